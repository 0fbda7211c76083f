// Host-side check of the evaluation planner (hg_internal.cuh): prints, for
// each query line "m tuned_value" read from stdin, the bucket and the plan
// chosen with that value stored in m's bucket ("-" for the cost model alone),
// and the block sizes the autotuner would time for that bucket with m as the
// largest size tuned.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "hg_internal.cuh"

int main(int argc, char **argv)
{
    // Planner inputs of a mixed context with n = 65536 on 152 SMs.
    const long long npad = argc > 1 ? atoll(argv[1]) : 65536;
    hg::PlanParams q{};
    q.tj = hg::kTJMixed;
    q.i_per_thread = hg::kIMixed;
    q.ntiles = npad / q.tj;
    q.pcap = 4 * npad > (1 << 20) ? 4 * npad : (1 << 20);
    q.grid = 3 * 152;
    q.tpi_force = 0;
    q.b_force = 0;
    q.c_tile = 2;
    q.c_item = 24;
    q.variants = 1;   // one mixed kernel, one i-particle per thread
    q.ipt1 = hg::kIMixed;
    q.grid1 = q.grid;
    q.weight1 = q.weight1_one = 100;
    long long m;
    int v;
    while (scanf("%lld %d", &m, &v) == 2) {
        for (int k = 0; k < hg::kTuneBuckets; ++k) q.tuned[k] = -1;
        const int b = hg::tune_bucket(m);
        const hg::Plan model = hg::make_plan(m, q);
        q.tuned[b] = (int16_t)v;
        const hg::Plan p = hg::make_plan(m, q);
        const hg::BatchKnobs kn = hg::batch_knobs(m, q);
        long long pts[3] = {0, 0, 0};
        int64_t pt[3];
        const int np = hg::tune_points(b, m, pt);   // this bucket's tuning sizes, m as the largest
        for (int k = 0; k < np; ++k) pts[k] = (long long)pt[k];
        printf("%d %d %lld %d %lld %d %d %d %d %d %d %d %lld %lld %lld\n", b, model.tpi,
               (long long)model.tiles_per_split, p.tpi, (long long)p.tiles_per_split, p.b, kn.w_log, kn.tpi_shift,
               p.variant, p.ti, model.variant, np, pts[0], pts[1], pts[2]);
    }
    return 0;
}
