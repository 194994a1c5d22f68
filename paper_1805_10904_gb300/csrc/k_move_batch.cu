// k_move_batch.cu -- the batch instantiation of the sweep kernels of k_move_impl.cuh
// (several graphs stacked into one CSR, each with its own 2W and phase controller).  It is a
// translation unit of its own so that it compiles in parallel with the one-graph kernels.
#include "k_move_impl.cuh"

namespace lv {

int launch_sweep_batch(const DevGraph &g, const PhaseState &st, const Bins &b, i64 tw, bool wide,
                       bool narrow, SweepStats *stats, unsigned *err, cudaStream_t s,
                       const LaunchCfg &lc, SweepTimers *tm, const BatchCtx &bc)
{
    return sweep_typed<true, false>(g, st, b, tw, wide, narrow, stats, err, s, lc, tm, bc);
}

}  // namespace lv
