// step_tiled.cu -- the temporal-blocking kernels (step_tiled.cuh) for Eq. 3 as
// printed, the host-side split of a grid into (chunk, strip) work items, and
// the launchers, which send the scheme options to step_tiled_opts.cu.
#include "step_tiled.cuh"

namespace flood {

// Row chunks for the (chunk, strip) work items of a grid of n_strips strips and
// ny rows on `resident` pipelines: the chunk count minimises the ticks of the
// busiest pipeline, (items per pipeline) x (chunk rows + 3K - 1), an item
// costing its rows plus 2K - 1 staged halo rows and the 2(K - 1) ticks by
// which level K lags level 1.
void tiled_split(int n_strips, int ny, int resident, int K, int *chunk_rows, int *blocks)
{
    static thread_local int memo[4] = {-1, -1, -1, -1}, memo_rows = 0;   // per thread: no race between handles
    if (memo[0] == n_strips && memo[1] == ny && memo[2] == resident && memo[3] == K) {
        const long long items = (long long)n_strips * ((ny + memo_rows - 1) / memo_rows);
        *chunk_rows = memo_rows;
        *blocks = (int)(items < resident ? items : resident);
        return;
    }
    long long best = -1;
    int best_rows = ny;
    const int max_chunks = (ny + 15) / 16;            // chunks of at least 16 rows
    for (int c = 1; c <= max_chunks; c++) {
        const int rows = (ny + c - 1) / c;
        const int chunks = (ny + rows - 1) / rows;
        const long long items = (long long)n_strips * chunks;
        const long long waves = (items + resident - 1) / resident;
        const long long ticks = waves * (rows + 3 * K - 1);
        if (best < 0 || ticks < best) {
            best = ticks;
            best_rows = rows;
        }
    }
    memo[0] = n_strips;
    memo[1] = ny;
    memo[2] = resident;
    memo[3] = K;
    memo_rows = best_rows;
    const long long items = (long long)n_strips * ((ny + best_rows - 1) / best_rows);
    *chunk_rows = best_rows;
    *blocks = (int)(items < resident ? items : resident);
}

// The same when the pipelines take their items from a counter as they come free:
// about eight items per pipeline, so that the ones that finish early take more
// and the launch ends evenly, of at least 24 K rows (an item costs its rows plus
// the 3K - 1 ticks of filling the pipeline); a grid that would get fewer than four
// such items per pipeline keeps the round-robin split.  Measured against fixed
// rows per item of 64 ... 384 on the fractal workload at 16384^2 (304 rows: 8
// items per pipeline) and 8192^2 (96 rows: 6.5), and against the round-robin
// split at 4096^2 and 2048^2.
void tiled_split_dynamic(int n_strips, int ny, int resident, int K, int *chunk_rows, int *blocks)
{
    const long long target = 8LL * resident;
    const long long chunks = (target + n_strips - 1) / n_strips;
    int rows = (int)((ny + chunks - 1) / chunks);
    const int min_rows = 24 * K;
    if (rows < min_rows) {
        rows = min_rows;
        if ((long long)n_strips * ((ny + rows - 1) / rows) < 4LL * resident) {
            tiled_split(n_strips, ny, resident, K, chunk_rows, blocks);
            return;
        }
    }
    const long long items = (long long)n_strips * ((ny + rows - 1) / rows);
    *chunk_rows = rows;
    *blocks = (int)(items < resident ? items : resident);
}

int tiled_items(const Geom &g, int chunk_rows, int k_steps)
{
    const int mode = (g.theta != 1.0 ? 1 : 0) | (g.friction != 0 ? 2 : 0);
    const int out = out_cols(k_steps, mode);
    const int n_strips = (g.nx + out - 1) / out;
    return n_strips * ((g.ny + chunk_rows - 1) / chunk_rows);
}

// Scheme mode of a grid: bit 0 theta weighting, bit 1 vector-norm friction.
static int tiled_mode(const Geom &g) { return (g.theta != 1.0 ? 1 : 0) | (g.friction != 0 ? 2 : 0); }

// step_tiled_opts.cu: the same launchers for modes 1..3.
cudaError_t launch_step_tiled_opts(const StepArgs<float> &a, int mode, cudaStream_t st);
cudaError_t launch_step_tiled_ensemble_opts(const StepArgs<float> *table, const int *base, int n, int total_items,
                                            int k_steps, int s0, int want_hmax, int *next_item, int mode,
                                            cudaStream_t st);

cudaError_t launch_step_tiled_ensemble(const StepArgs<float> *table, const int *base, int n, int total_items,
                                       int k_steps, int s0, int want_hmax, int *next_item, int mode, cudaStream_t st)
{
    if (mode != 0)
        return launch_step_tiled_ensemble_opts(table, base, n, total_items, k_steps, s0, want_hmax, next_item, mode,
                                               st);
    return launch_tiled_ensemble_mode<0>(table, base, n, total_items, k_steps, s0, want_hmax, next_item, st);
}

cudaError_t launch_step_tiled(const StepArgs<float> &a, cudaStream_t st)
{
    const int mode = tiled_mode(a.geo);
    if (mode != 0) return launch_step_tiled_opts(a, mode, st);
    return launch_tiled_mode<0>(a, st);
}

}  // namespace flood

#include "flood.h"

extern "C" flood_status flood_debug_tiled_split(int32_t nx, int32_t ny, int32_t k_steps, int32_t mode,
                                                int32_t resident, int32_t *chunk_rows, int32_t *blocks,
                                                int32_t *n_items)
{
    using namespace flood;
    if (nx < 1 || ny < 1 || !(k_steps >= 1 && (k_steps <= 4 || k_steps == 8)) || mode < 0 || mode > 3 ||
        resident < 1 || !chunk_rows || !blocks || !n_items)
        return FLOOD_ERR_ARG;
    const int out = out_cols(k_steps, mode);
    const int n_strips = (nx + out - 1) / out;
    int rows = 0, b = 0;
    tiled_split_dynamic(n_strips, ny, resident, k_steps, &rows, &b);
    const long long items = (long long)n_strips * ((ny + rows - 1) / rows);
    if (items > 0x7fffffffLL) return FLOOD_ERR_ARG;
    *chunk_rows = rows;
    *blocks = b;
    *n_items = (int32_t)items;
    return FLOOD_OK;
}
