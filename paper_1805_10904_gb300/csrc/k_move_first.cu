// k_move_first.cu -- the first sweep of a phase (k_move_impl.cuh, FIRST = true): bins 0-9
// score row entries without tables, for one graph and for a batch of graphs.
#include "k_move_impl.cuh"

namespace lv {

int launch_sweep_first(const DevGraph &g, const PhaseState &st, const Bins &b, i64 tw, bool wide,
                       bool narrow, SweepStats *stats, unsigned *err, cudaStream_t s,
                       const LaunchCfg &lc, SweepTimers *tm, const BatchCtx &bc)
{
    if (bc.vg) return sweep_typed<true, true>(g, st, b, tw, wide, narrow, stats, err, s, lc, tm, bc);
    return sweep_typed<false, true>(g, st, b, tw, wide, narrow, stats, err, s, lc, tm, bc);
}

}  // namespace lv
