// The autotuner of the batched launch. A process-wide table maps a method (input
// format, storage, radius, levels, iterations, normalisation, variant) and a size class
// (round(log2(mean level-0 pixels per pair))) to a Tuning: window-sum strategy, I2
// staging, and either phase launches or the persistent launch at some resident blocks
// per SM. of_compute_batch and the serving loop read it; of_autotune_batch fills it by
// timing every candidate on the caller's own batch.
#include <math.h>
#include <string.h>

#include <array>
#include <map>
#include <mutex>
#include <vector>

#include "of_engine.h"
#include "of_internal.cuh"

namespace of {

namespace {

using Key = std::array<int, 8>;

std::mutex g_tune_mu;
std::map<Key, Tuning> g_table;

Key key_of(const of_plan &m, int size_class)
{
    return {m.in_format,
            m.storage,
            m.radius,
            m.levels,
            m.iterations,
            (m.flags & OF_FLAG_ZNSSD) ? 1 : 0,
            (m.flags & OF_FLAG_I1GRAD) ? 1 : 0,   // the variant runs other kernels
            size_class};
}

bool valid(const Tuning &t)
{
    return t.generic_sums >= 0 && t.generic_sums <= 1 && t.stage_i2 >= 0 && t.stage_i2 <= 1 && t.blocks_per_sm >= 0 &&
           t.blocks_per_sm <= 64 && t.phased >= 0 && t.phased <= 1 && !(t.generic_sums && t.stage_i2) &&
           !(t.phased && t.blocks_per_sm) && t.prefetch >= 0 && t.prefetch <= 16 &&
           (t.tile_h == 0 || t.tile_h == LK_TH || (t.tile_h == ALT_TH && t.phased && !t.generic_sums)) &&
           t.branches >= 0 && t.branches <= 4 && (t.branches <= 1 || t.phased) && t.fusion >= 0 && t.fusion <= 2 &&
           (t.fusion <= 1 || (t.phased && !t.generic_sums && (t.tile_h == 0 || t.tile_h == LK_TH))) &&
           (t.strip == 0 || t.strip == 1 || t.strip == 2 || t.strip == 4) &&
           (t.strip <= 1 || (t.phased && !t.generic_sums));
}

void to_c(const Tuning &t, float ms, of_tuning *o)
{
    o->generic_sums = t.generic_sums;
    o->stage_i2 = t.stage_i2;
    o->blocks_per_sm = t.blocks_per_sm;
    o->phased = t.phased;
    o->prefetch = t.prefetch;
    o->tile_h = t.tile_h ? t.tile_h : LK_TH;
    o->branches = t.branches ? t.branches : 1;
    o->fusion = t.fusion ? t.fusion : 1;
    o->strip = tuning_strip(t);
    o->ms = ms;
}

}  // namespace

Tuning tuning_for(const of_plan &method, int size_class)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_table.find(key_of(method, size_class));
    return it == g_table.end() ? Tuning() : it->second;
}

int batch_size_class(int32_t n, const of_handle *hs)
{
    double px = 0.0;
    int m = 0;
    for (int i = 0; i < n; ++i)
        if (hs[i]) {
            px += (double)hs[i]->lay.H[0] * hs[i]->lay.W[0];
            ++m;
        }
    return m ? (int)lround(log2(px / m)) : 0;
}

}  // namespace of

using namespace of;

extern "C" {

int of_batch_size_class(int32_t n, const of_handle *hs, int32_t *size_class)
{
    if (n < 1 || !hs || !size_class) return OF_EINVAL;
    for (int i = 0; i < n; ++i)
        if (!hs[i]) return OF_EINVAL;
    *size_class = batch_size_class(n, hs);
    return OF_OK;
}

int of_tuning_get(const of_plan *method, int32_t size_class, of_tuning *t)
{
    if (of_plan_validate(method) != OF_OK || !t) return OF_EINVAL;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_table.find(key_of(*method, size_class));
    if (it == g_table.end()) return OF_ESTATE;
    to_c(it->second, 0.0f, t);
    return OF_OK;
}

int of_tuning_set(const of_plan *method, int32_t size_class, const of_tuning *t)
{
    if (of_plan_validate(method) != OF_OK || !t) return OF_EINVAL;
    Tuning v;
    v.generic_sums = t->generic_sums;
    v.stage_i2 = t->stage_i2;
    v.blocks_per_sm = t->blocks_per_sm;
    v.phased = t->phased;
    v.prefetch = t->prefetch;
    v.tile_h = t->tile_h == LK_TH ? 0 : t->tile_h;
    v.branches = t->branches == 1 ? 0 : t->branches;
    v.fusion = t->fusion == 1 ? 0 : t->fusion;
    v.strip = t->strip == 4 ? 0 : t->strip;
    if (!valid(v)) return OF_EINVAL;
    if (v.fusion == 2 && !radius_specialised(method->radius)) return OF_EINVAL;   // fixed-radius kernels only
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_table[key_of(*method, size_class)] = v;
    return OF_OK;
}

int of_tuning_clear(void)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_table.clear();
    return OF_OK;
}

int of_autotune_batch(int32_t n, const of_handle *hs, const void *const *I1s, const void *const *I2s,
                      float *const *us, float *const *vs, of_stream_t stream, int32_t reps, of_tuning *best,
                      of_tuning *results, int32_t max_results, int32_t *n_results)
{
    if (n < 1 || !hs || !I1s || reps < 1 || reps > 1000 || max_results < 0 || (max_results > 0 && !results))
        return OF_EINVAL;
    for (int i = 0; i < n; ++i)
        if (!hs[i] || !I1s[i]) return OF_EINVAL;   // repeated runs must not change which pyramid is reused
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const of_plan &p0 = hs[0]->plan;
    // candidates: the grouped fixed-radius sums (gathered or staged I2) when the radius
    // has a specialised kernel, the per-output sums of the run-time-radius kernel; each
    // as phase launches with no L2 prefetch or one 1 or 3 blocks per SM ahead (the grouped
    // sums also with the other tile height; without prefetch also as two concurrent
    // launch sequences over halves of the batch; the grouped sums in strips of 4 tiles per
    // block, staged at the default tile height also one tile per block), and as the
    // persistent launch at full occupancy and at 2 and 1 blocks per SM
    std::vector<Tuning> cand;
    const int occ[6] = {-1, -2, -3, 0, 2, 1};   // < 0: phase launches with prefetch pf_of[-1 - b]
    const int pf_of[3] = {0, 1, 3};
    const bool variant = (p0.flags & OF_FLAG_I1GRAD) != 0;
    for (int gs = radius_specialised(p0.radius) ? 0 : 1; gs <= 1; ++gs)
        for (int sg = 0; sg <= (gs ? 0 : 1); ++sg)
            for (int th = 0; th <= ((gs || variant) ? 0 : 1); ++th)
                for (int b : occ) {
                    if (variant && (b >= 0 || sg)) continue;   // phase launches, gathered taps only
                    if (th && b >= 0) continue;                // the persistent launch has one tile height
                    if (sg && b >= 0) continue;                // and gathers its taps
                    Tuning t;
                    t.generic_sums = gs;
                    t.stage_i2 = sg;
                    t.phased = b < 0 ? 1 : 0;
                    t.blocks_per_sm = b < 0 ? 0 : b;
                    t.prefetch = b < 0 ? pf_of[-1 - b] : 0;
                    t.tile_h = th ? ALT_TH : 0;
                    t.strip = (t.phased && !gs) ? 0 : 1;
                    cand.push_back(t);
                    if (t.phased && t.prefetch == 0 && n > 1) {
                        t.branches = 2;
                        cand.push_back(t);
                    }
                    if (t.phased && !gs && sg && !th && t.prefetch == 0) {
                        // one tile per block (every tile its own stage 1 and horizontal pass)
                        t.strip = 1;
                        t.branches = 0;
                        cand.push_back(t);
                        if (n > 1) {
                            t.branches = 2;
                            cand.push_back(t);
                        }
                    }
                }
    // iteration fusion depth 2 (grouped sums, default tile height, phase launches), in one
    // and in two concurrent sequences
    if (radius_specialised(p0.radius) && !variant)
        for (int nb = 1; nb <= (n > 1 ? 2 : 1); ++nb) {
            Tuning t;
            t.fusion = 2;
            t.branches = nb > 1 ? nb : 0;
            cand.push_back(t);
        }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return OF_ECUDA;
    }
    int rc = OF_OK, nres = 0, ibest = -1;
    float best_ms = 0.0f;
    for (size_t c = 0; c < cand.size() && rc == OF_OK; ++c) {
        // one untimed launch (captures the graph), then reps timed launches
        if ((rc = run_batch(n, hs, I1s, I2s, us, vs, st, cand[c])) != OF_OK) break;
        if (cudaEventRecord(e0, st) != cudaSuccess) { rc = OF_ECUDA; break; }
        for (int k = 0; k < reps && rc == OF_OK; ++k) rc = run_batch(n, hs, I1s, I2s, us, vs, st, cand[c]);
        if (rc != OF_OK) break;
        float ms = 0.0f;
        if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            rc = OF_ECUDA;
            break;
        }
        ms /= (float)reps;
        for (int i = 0; i < n; ++i) {   // a device-side failure (a timed-out wait) disqualifies the run
            const int s = of_sync_status(hs[i]);
            if (s != OF_OK) rc = s;
        }
        if (rc != OF_OK) break;
        if (nres < max_results) to_c(cand[c], ms, &results[nres++]);
        if (ibest < 0 || ms < best_ms) {
            ibest = (int)c;
            best_ms = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (n_results) *n_results = nres;
    if (rc != OF_OK) return rc;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_table[key_of(p0, batch_size_class(n, hs))] = cand[ibest];
    }
    if (best) to_c(cand[ibest], best_ms, best);
    return OF_OK;
}

}  // extern "C"
