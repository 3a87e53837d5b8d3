// autotune.cpp -- chooses the launch configuration of the coarse step by
// timing candidates on scratch states of the caller's mesh, regions and
// initial state.
//
// Knobs: threads per block, the kernel path (three launches per right-hand
// side or fused tiles), programmatic dependent launch, the L2
// eviction-priority hints, the schedule of the coarse phases (which run as a
// concurrent graph branch), and (optionally) the cell ordering in the bands.
// None of them changes a result bit (each element's arithmetic is the same
// in every configuration), so the choice is purely a matter of time.
#include <algorithm>
#include <cmath>
#include <vector>

#include "../../include/lts.h"
#include "lts_error.h"
#include "lts_internal.h"
#include "lts_objects.h"

using namespace lts;

namespace {

struct Candidate {
    int block, path, pdl, no_l2, serial;   // serial: the coarse schedule
    double ms = INFINITY;
    int occ = 0;                           // ring occupancy variant
    int ept = 0;                           // elements per thread (0: the base's)
};

lts_params apply(const lts_params& base, const Candidate& c) {
    lts_params p = base;
    p.block_size = c.block;
    p.kernel_path = c.path;
    p.pdl = c.pdl;
    p.no_l2_hints = c.no_l2;
    p.coarse_schedule = c.serial;
    p.ring_occupancy = c.occ;
    if (c.ept) p.elems_per_thread = c.ept;
    p.use_graph = 1;
    p.profile = 0;
    p.stream = nullptr;
    return p;
}

// Milliseconds per coarse step of one configuration (3 warm-up steps, then
// `steps` steps between two events on the state's stream); INFINITY when the
// configuration cannot be built for this mesh (e.g. tiles that do not fit).
int time_config(lts_mesh m, lts_regions r, const double* h0, const double* u0, const lts_params& p,
                int steps, double* ms) {
    *ms = INFINITY;
    lts_state s = nullptr;
    int rc = lts_state_create(m, r, h0, u0, &p, &s);
    if (rc == LTS_EINVAL) return LTS_OK;   // not available for this mesh: skipped
    if (rc != LTS_OK) return rc;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    if (err == cudaSuccess) {
        rc = lts_step(s, 3);
        if (rc == LTS_OK) err = cudaEventRecord(e0, s->stream);
        if (rc == LTS_OK && err == cudaSuccess) rc = lts_step(s, steps);
        if (rc == LTS_OK && err == cudaSuccess) err = cudaEventRecord(e1, s->stream);
        if (rc == LTS_OK && err == cudaSuccess) err = cudaEventSynchronize(e1);
        float t = 0.f;
        if (rc == LTS_OK && err == cudaSuccess) err = cudaEventElapsedTime(&t, e0, e1);
        if (rc == LTS_OK && err == cudaSuccess) *ms = t / steps;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    lts_state_destroy(s);
    if (rc != LTS_OK) return rc;
    if (err != cudaSuccess) return set_error(LTS_ECUDA, "autotune timing: %s", cudaGetErrorString(err));
    return LTS_OK;
}

}  // namespace

extern "C" int lts_autotune(lts_mesh m, lts_regions r, const double* h0, const double* u0,
                            const lts_params* base, int32_t steps, int32_t flags, lts_params* best,
                            lts_tune_report* rep) {
    if (!m || !r || !h0 || !u0 || !base || !best) return set_error(LTS_EINVAL, "null argument");
    if (steps < 1 || steps > 100000) return set_error(LTS_EINVAL, "steps must be in [1, 100000]");
    std::vector<Candidate> cands;
    const bool lts3 = base->mode == LTS_MODE_LTS && r->r.order == 3;
    const bool lts = base->mode == LTS_MODE_LTS;
    const bool fused_ok = base->mode == LTS_MODE_SSPRK3 || lts3;
    // three-launch path: every combination; fused tiles (one block per
    // 256-cell tile): with PDL, concurrent (the fused plans branch Step 4
    // only) or serial
    // coarse schedules: LTS2 has no far Steps 1/2 (its FAR is the Step-4
    // branch), the global SSP-RK modes have no coarse phases at all
    std::vector<int> scheds = {LTS_COARSE_FAR};
    if (lts3) scheds = {LTS_COARSE_FAR, LTS_COARSE_STEP4, LTS_COARSE_SERIAL};
    else if (lts) scheds = {LTS_COARSE_FAR, LTS_COARSE_SERIAL};
    for (int block : {128, 256})
        for (int pdl = 1; pdl >= 0; --pdl)
            for (int no_l2 = 0; no_l2 <= 1; ++no_l2)
                for (int sched : scheds) cands.push_back({block, 0, pdl, no_l2, sched});
    if (fused_ok)
        for (int no_l2 = 0; no_l2 <= 1; ++no_l2)
            for (int sched : {LTS_COARSE_FAR, LTS_COARSE_SERIAL})
                if (lts3 || sched == LTS_COARSE_FAR) cands.push_back({256, 1, 1, no_l2, sched});
    // every candidate once, then the three fastest twice more (best of three)
    for (Candidate& c : cands) {
        int rc = time_config(m, r, h0, u0, apply(*base, c), steps, &c.ms);
        if (rc != LTS_OK) return rc;
    }
    std::vector<size_t> order(cands.size());
    for (size_t k = 0; k < order.size(); ++k) order[k] = k;
    std::sort(order.begin(), order.end(), [&](size_t a, size_t b) { return cands[a].ms < cands[b].ms; });
    const size_t top = std::min<size_t>(3, order.size());
    for (int rep_k = 0; rep_k < 2; ++rep_k)
        for (size_t k = 0; k < top; ++k) {
            Candidate& c = cands[order[k]];
            double ms = INFINITY;
            int rc = time_config(m, r, h0, u0, apply(*base, c), steps, &ms);
            if (rc != LTS_OK) return rc;
            c.ms = std::min(c.ms, ms);
        }
    const Candidate* win = &cands[order[0]];
    for (size_t k = 0; k < top; ++k)
        if (cands[order[k]].ms < win->ms) win = &cands[order[k]];
    if (!std::isfinite(win->ms)) return set_error(LTS_EINVAL, "no configuration could be built");
    double default_ms = INFINITY;
    for (const Candidate& c : cands)
        if (c.block == 256 && c.path == 0 && c.pdl == 1 && c.no_l2 == 0 && c.serial == LTS_COARSE_FAR)
            default_ms = c.ms;
    // the FP32 ring-pass occupancy variants with the winning configuration;
    // layered and multi-region states launch other kernels, so they have none
    Candidate occ_best = *win;
    std::vector<Candidate> occ_tried;
    const bool multi = r->r.nreg > 1 && base->mode == LTS_MODE_LTS;
    if (base->precision == LTS_FP32 && win->path == 0 && base->layers <= 1 && !multi) {
        for (int occ : {6, 8}) {
            Candidate c = *win;
            c.occ = occ;
            for (int rep_k = 0; rep_k < 2; ++rep_k) {
                double ms = INFINITY;
                int rc = time_config(m, r, h0, u0, apply(*base, c), steps, &ms);
                if (rc != LTS_OK) return rc;
                c.ms = rep_k == 0 ? ms : std::min(c.ms, ms);
            }
            occ_tried.push_back(c);
            if (c.ms < occ_best.ms) occ_best = c;
        }
    }
    win = &occ_best;
    // the other number of elements per thread of the vertex and edge launches
    const int ept0 = base->elems_per_thread ? base->elems_per_thread : LTS_DEFAULT_EPT;
    Candidate ept_best = *win;
    std::vector<Candidate> ept_tried;
    if (win->path == 0 && base->layers <= 1 && !multi) {
        Candidate c = *win;
        c.ept = 3 - ept0;
        for (int rep_k = 0; rep_k < 2; ++rep_k) {
            double ms = INFINITY;
            int rc = time_config(m, r, h0, u0, apply(*base, c), steps, &ms);
            if (rc != LTS_OK) return rc;
            c.ms = rep_k == 0 ? ms : std::min(c.ms, ms);
        }
        ept_tried.push_back(c);
        if (c.ms < ept_best.ms) ept_best = c;
    }
    win = &ept_best;
    *best = apply(*base, *win);
    best->stream = base->stream;
    double best_ms = win->ms;
    int ordering = r->r.ordering, tried_orderings = 1;
    const int ordering0 = ordering;
    double other_ms = INFINITY;
    if ((flags & LTS_TUNE_ORDERING) && r->ref.load() == 1) {
        // the other cell ordering with the winning launch configuration
        const int other = 1 - ordering;
        int rc = lts_regions_ordering(r, other);
        if (rc != LTS_OK) return rc;
        double ms = INFINITY;
        rc = time_config(m, r, h0, u0, apply(*base, *win), steps, &ms);
        if (rc != LTS_OK) return rc;
        tried_orderings = 2;
        other_ms = ms;
        if (ms < best_ms) {
            best_ms = ms;
            ordering = other;
        } else {
            rc = lts_regions_ordering(r, ordering);
            if (rc != LTS_OK) return rc;
        }
    }
    if (rep) {
        rep->candidates = static_cast<int32_t>(cands.size() + occ_tried.size() + ept_tried.size()) +
                          (tried_orderings - 1);
        rep->best_ms = best_ms;
        rep->default_ms = default_ms;
        rep->ordering = ordering;
        // every candidate ran with the initial ordering; the extra trial with the other one
        int n = 0;
        for (const Candidate& c : cands) {
            if (n >= 32) break;
            rep->entry[n++] = {c.block, c.path, c.pdl, 1 - c.no_l2, c.serial, ordering0, 0, ept0, c.ms};
        }
        for (const Candidate& c : occ_tried)
            if (n < 32)
                rep->entry[n++] = {c.block, c.path, c.pdl, 1 - c.no_l2, c.serial, ordering0, c.occ, ept0, c.ms};
        for (const Candidate& c : ept_tried)
            if (n < 32)
                rep->entry[n++] = {c.block, c.path, c.pdl, 1 - c.no_l2, c.serial, ordering0, c.occ, c.ept, c.ms};
        if (tried_orderings == 2 && n < 32)
            rep->entry[n++] = {win->block, win->path, win->pdl, 1 - win->no_l2, win->serial, 1 - ordering0,
                               win->occ, win->ept ? win->ept : ept0, other_ms};
    }
    return LTS_OK;
}
