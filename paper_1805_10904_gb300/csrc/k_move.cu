// k_move.cu -- the one-graph instantiation of the sweep kernels of k_move_impl.cuh, the
// sweep entry point, and the shared-memory / cluster capability probes.
#include "k_move_impl.cuh"

namespace lv {

template <int CL>
static bool cluster_fits(size_t smem)
{
    auto kernel = k_move_cluster<CL, int32_t, i64, unsigned int, false>;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (CL > 8) cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(CL, 1, 1);
    cfg.blockDim = dim3(1024, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int maxc = 0;
    const cudaError_t e = cudaOccupancyMaxActiveClusters(&maxc, kernel, &cfg);
    cudaGetLastError();
    return e == cudaSuccess && maxc >= 1;
}

void probe_cluster_support(size_t smem, bool ok[4])
{
    ok[0] = cluster_fits<2>(smem);
    ok[1] = cluster_fits<4>(smem);
    ok[2] = cluster_fits<8>(smem);
    ok[3] = cluster_fits<16>(smem);
}

size_t shared_table_bytes(int log2cap, bool narrow)
{
    return narrow ? table_bytes<unsigned int>(log2cap) : table_bytes<u64>(log2cap);
}

// The other instantiations, each a translation unit of its own so that they compile in
// parallel: k_move_batch.cu (a batch of graphs), k_move_first.cu (first sweep of a phase,
// one graph and a batch).
int launch_sweep_batch(const DevGraph &g, const PhaseState &st, const Bins &b, i64 tw, bool wide,
                       bool narrow, SweepStats *stats, unsigned *err, cudaStream_t s,
                       const LaunchCfg &lc, SweepTimers *tm, const BatchCtx &bc);
int launch_sweep_first(const DevGraph &g, const PhaseState &st, const Bins &b, i64 tw, bool wide,
                       bool narrow, SweepStats *stats, unsigned *err, cudaStream_t s,
                       const LaunchCfg &lc, SweepTimers *tm, const BatchCtx &bc);

int launch_sweep(const DevGraph &g, const PhaseState &st, const Bins &b, i64 tw, bool wide,
                 bool narrow, bool first, SweepStats *stats, unsigned *err, cudaStream_t s,
                 const LaunchCfg &lc, SweepTimers *tm, const BatchCtx &bc)
{
    if (first) return launch_sweep_first(g, st, b, tw, wide, narrow, stats, err, s, lc, tm, bc);
    if (bc.vg) return launch_sweep_batch(g, st, b, tw, wide, narrow, stats, err, s, lc, tm, bc);
    return sweep_typed<false, false>(g, st, b, tw, wide, narrow, stats, err, s, lc, tm, bc);
}

}  // namespace lv
