// ensemble.cpp -- several independent meshes advanced together: one launch
// per phase of the coarse step for all members.
//
// Every member is an lts_state of its own mesh, regions, M and dt.  The
// ensemble concatenates the members' band-ordered device tables and states
// into one packed index space (member after member; inside a member the
// band order of its regions), builds each member's three-launch plan of
// Algorithm 2.2 (or 2.1) against the packed buffers, and merges the plans
// launch by launch: launches with the same phase key (step, substep, stage,
// kind) become one launch whose segment list holds every member's segments.
// A member with a smaller M simply has no segments in the later substeps.
// The segment lists live in device memory; each block of a launch finds its
// segment by a binary search (kernel_phase_table), so a launch may carry any
// number of members.  Each
// member's cells see exactly the arithmetic of its stand-alone step.
#include <algorithm>
#include <cstring>
#include <map>
#include <memory>
#include <new>
#include <vector>

#include "../../include/lts.h"
#include "lts_error.h"
#include "lts_internal.h"
#include "lts_objects.h"
#include "regions.h"

using namespace lts;

struct lts_ensemble_s {
    std::vector<lts_state_s*> members;
    std::vector<double> t0;           // member clocks when the ensemble was made
    std::vector<int64_t> steps0;
    KernelConfig kc{};
    size_t tsz = 4;
    double g = 9.81;
    int NC = 0, NE = 0, NV = 0, MAXE = 0;
    std::vector<int> offC, offE, offV;          // member offsets in the packed arrays
    std::vector<int> oI1c, oIc, oI1e, oIe;      // member offsets in the compact arrays
    DeviceArena arena;
    Tables<float> t32{};
    Tables<double> t64{};
    const void* tables = nullptr;
    SV buf[4];
    SV P1c, P1e, P2c, P2e;
    void* acc_c[3] = {};
    void* acc_e[3] = {};
    void* q = nullptr;
    void* ring_c = nullptr;
    void* ring_k = nullptr;
    void* q_side = nullptr;       // intermediates of the concurrent far-coarse branch
    void* ring_c_side = nullptr;
    void* ring_k_side = nullptr;
    int* flag = nullptr;
    std::vector<TableLaunch> plan[2];
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t capture_stream = nullptr, capture_side = nullptr, side_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // member I/O is ordered against the ensemble's stream by events, not by
    // host synchronisation; the shared error flag is read into pinned memory
    cudaEvent_t ev_io = nullptr;
    int* flag_host = nullptr;
    int parity = 0;
    int64_t steps = 0;
    int launches = 0;
    int segments = 0;
    double bytes[NKINDS] = {};
    ~lts_ensemble_s() {
        // a caller's stream may already be gone: only the library's own is
        // waited for (every flag copy into pinned memory completes inside
        // the lts_ensemble_read that issued it)
        if (own_stream && stream) cudaStreamSynchronize(stream);
        for (auto& e : exec)
            if (e) cudaGraphExecDestroy(e);
        if (own_stream && stream) cudaStreamDestroy(stream);
        if (capture_stream) cudaStreamDestroy(capture_stream);
        if (capture_side) cudaStreamDestroy(capture_side);
        if (side_stream) cudaStreamDestroy(side_stream);
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        if (ev_io) cudaEventDestroy(ev_io);
        if (flag_host) cudaFreeHost(flag_host);
    }
};

namespace {

// Union of the members' band-ordered tables, indices shifted by the member
// offsets.  Slot-major cell arrays are re-strided to the total cell count;
// slots past a member's own maxEdges repeat slot 0 (the padding rule of the
// single-mesh tables), so every slot may still be loaded unconditionally.
template <class T>
int build_union_tables(lts_ensemble_s* E, Tables<T>& t) {
    const size_t NC = E->NC, NE = E->NE, NV = E->NV, W = slot_rows(E->MAXE);
    std::vector<uint8_t> cn(NC);
    std::vector<int> se(W * NC), sn(W * NC), sv(W * NC);
    std::vector<T> snl(W * NC), sR(W * NC), sK(W * NC), rA(NC), b(NC);
    std::vector<double> sK64(W * NC), area(NC), bd(NC);
    std::vector<int> ec0(NE), ec1(NE);
    std::vector<uint32_t> ep(NE);
    std::vector<T> rdc(NE), db(NE);
    std::vector<int> vc(3 * NV), ve(3 * NV);
    std::vector<T> vk(3 * NV), vd(3 * NV), f(NV);
    for (size_t m = 0; m < E->members.size(); ++m) {
        const HostMesh& hm = E->members[m]->reg->mesh->m;
        const RegionsHost& r = E->members[m]->reg->r;
        CoefTables<T> co;
        coefficient_tables<T>(hm, r, co);
        const size_t nC = hm.nC, nE = hm.nE, nV = hm.nV, w = hm.maxE;
        const size_t oc = E->offC[m], oe = E->offE[m], ov = E->offV[m];
        for (size_t c = 0; c < nC; ++c) {
            cn[oc + c] = r.cn[c];
            rA[oc + c] = co.rA[c];
            b[oc + c] = co.b[c];
            area[oc + c] = co.area[c];
            bd[oc + c] = co.bd[c];
        }
        for (size_t j = 0; j < W; ++j) {
            const size_t jj = j < w ? j : 0;
            for (size_t c = 0; c < nC; ++c) {
                const size_t src = jj * nC + c, dst = j * NC + oc + c;
                se[dst] = r.se[src] + static_cast<int>(oe);
                sn[dst] = r.sn[src] + static_cast<int>(oc);
                sv[dst] = r.sv[src] + static_cast<int>(ov);
                snl[dst] = co.snl[src];
                sR[dst] = co.sR[src];
                sK[dst] = co.sK[src];
                sK64[dst] = co.sK64[src];
            }
        }
        for (size_t e = 0; e < nE; ++e) {
            ec0[oe + e] = r.ec0[e] + static_cast<int>(oc);
            ec1[oe + e] = r.ec1[e] + static_cast<int>(oc);
            ep[oe + e] = r.ep[e];
            rdc[oe + e] = co.rdc[e];
            db[oe + e] = co.db[e];
        }
        for (size_t k = 0; k < 3; ++k)
            for (size_t v = 0; v < nV; ++v) {
                vc[k * NV + ov + v] = r.vc[k * nV + v] + static_cast<int>(oc);
                ve[k * NV + ov + v] = r.ve[k * nV + v] + static_cast<int>(oe);
                vk[k * NV + ov + v] = co.vk[k * nV + v];
                vd[k * NV + ov + v] = co.vd[k * nV + v];
            }
        for (size_t v = 0; v < nV; ++v) f[ov + v] = co.f[v];
    }
    cudaError_t err = cudaSuccess;
    auto up = [&](const auto& v) { return E->arena.upload(v, err); };
    t = Tables<T>{};
    t.nC = E->NC;
    t.nE = E->NE;
    t.nV = E->NV;
    t.maxE = E->MAXE;
    t.cn = up(cn);
    t.se = up(se);
    t.sn = up(sn);
    t.sv = up(sv);
    t.snl = up(snl);
    t.sR = up(sR);
    t.sK = up(sK);
    {
        std::vector<int4> sidx;
        std::vector<float2> scf;
        pack_ring_slots<T>(se, sn, sv, snl, sR, sK, sidx, scf);
        t.sidx = up(sidx);
        t.scf = sizeof(T) == 4 ? up(scf) : nullptr;
    }
    {
        std::vector<int4> erow, vri;
        std::vector<float4> vrd, vrk;
        pack_edge_vertex_rows<T>(ec0, ec1, ep, rdc, vc, ve, vd, vk, f, erow, vri, vrd, vrk);
        t.erow = up(erow);
        t.vri = up(vri);
        t.vrd = sizeof(T) == 4 ? up(vrd) : nullptr;
        t.vrk = sizeof(T) == 4 ? up(vrk) : nullptr;
    }
    t.rA = up(rA);
    t.b = up(b);
    t.ec0 = up(ec0);
    t.ec1 = up(ec1);
    t.ep = up(ep);
    t.rdc = up(rdc);
    t.db = up(db);
    const int* dvc = up(vc);
    const int* dve = up(ve);
    const T* dvk = up(vk);
    const T* dvd = up(vd);
    t.f = up(f);
    t.area = up(area);
    t.bd = up(bd);
    t.sK64 = up(sK64);
    if (err != cudaSuccess)
        return set_error(err == cudaErrorMemoryAllocation ? LTS_ENOMEM : LTS_ECUDA, "ensemble tables: %s",
                         cudaGetErrorString(err));
    t.vc0 = dvc; t.vc1 = dvc + NV; t.vc2 = dvc + 2 * NV;
    t.ve0 = dve; t.ve1 = dve + NV; t.ve2 = dve + 2 * NV;
    t.vk0 = dvk; t.vk1 = dvk + NV; t.vk2 = dvk + 2 * NV;
    t.vd0 = dvd; t.vd1 = dvd + NV; t.vd2 = dvd + 2 * NV;
    return LTS_OK;
}

int alloc_state(lts_ensemble_s* E) {
    const size_t T = E->tsz;
    const bool comp = E->kc.comp;
    cudaError_t err = cudaSuccess;
    auto A = [&](size_t n) { return E->arena.alloc(n * T, err); };
    for (SV& x : E->buf) {
        x.hh = A(E->NC);
        x.uh = A(E->NE);
        if (comp) {
            x.hl = A(E->NC);
            x.ul = A(E->NE);
        }
    }
    const size_t n = E->members.size();
    const size_t nI1c = E->oI1c[n], nIc = E->oIc[n], nI1e = E->oI1e[n], nIe = E->oIe[n];
    for (SV* p : {&E->P1c, &E->P2c}) {
        p->hh = A(nI1c);
        if (comp) p->hl = A(nI1c);
    }
    for (SV* p : {&E->P1e, &E->P2e}) {
        p->uh = A(nI1e);
        if (comp) p->ul = A(nI1e);
    }
    for (int k = 0; k < 3; ++k) {
        E->acc_c[k] = A(nIc);
        E->acc_e[k] = A(nIe);
    }
    E->q = A(E->NV);
    E->ring_c = A(static_cast<size_t>(E->MAXE) * E->NC);
    E->ring_k = A(E->NC);
    E->q_side = A(E->NV);
    E->ring_c_side = A(static_cast<size_t>(E->MAXE) * E->NC);
    E->ring_k_side = A(E->NC);
    E->flag = static_cast<int*>(E->arena.alloc(sizeof(int), err));
    if (err != cudaSuccess)
        return set_error(err == cudaErrorMemoryAllocation ? LTS_ENOMEM : LTS_ECUDA, "ensemble state: %s",
                         cudaGetErrorString(err));
    CUDA_TRY(cudaDeviceSynchronize());   // the zero fills ran on the legacy stream
    return LTS_OK;
}

// Moves a member segment into the packed index space: its element range by
// the member's offset of that element kind, and every base that indexes a
// compact array so that (packed index - base) is the member's position in
// the packed compact array.
SegDesc place(const lts_ensemble_s* E, size_t m, SegDesc s) {
    const int off = s.elem == ELEM_CELL ? E->offC[m] : s.elem == ELEM_EDGE ? E->offE[m] : E->offV[m];
    auto coff = [&](int fam) {
        const bool cell = s.elem == ELEM_CELL;
        if (fam == FAM_I1) return cell ? E->oI1c[m] : E->oI1e[m];
        return cell ? E->oIc[m] : E->oIe[m];
    };
    s.begin += off;
    s.end += off;
    if (s.cfam != FAM_FULL) s.base += off - coff(s.cfam);
    if (s.cfam2 != FAM_FULL) s.base2 += off - coff(s.cfam2);
    return s;
}

// Host check of a placed segment: its element range lies inside member m's
// slice, and every compact index it forms lies inside the member's part of
// that compact array.
bool placed_in_bounds(const lts_ensemble_s* E, size_t m, const SegDesc& s) {
    const std::vector<int>& off = s.elem == ELEM_CELL ? E->offC : s.elem == ELEM_EDGE ? E->offE : E->offV;
    if (s.begin < off[m] || s.end > off[m + 1] || s.begin > s.end) return false;
    auto fam_ok = [&](int fam, int base) {
        if (fam == FAM_FULL) return true;
        if (s.elem == ELEM_VERT) return false;
        const bool cell = s.elem == ELEM_CELL;
        const std::vector<int>& o = fam == FAM_I1 ? (cell ? E->oI1c : E->oI1e) : (cell ? E->oIc : E->oIe);
        return s.begin - base >= o[m] && s.end - base <= o[m + 1];
    };
    return fam_ok(s.cfam, s.base) && fam_ok(s.cfam2, s.base2);
}

int build_plan(lts_ensemble_s* E, int parity, int nsm) {
    std::vector<std::vector<LaunchDesc>> plans;
    for (size_t m = 0; m < E->members.size(); ++m) {
        lts_state_s* S = E->members[m];
        // a view of the member whose buffers are the packed ones
        lts_state_s F;
        F.reg = S->reg;
        F.p = S->p;
        F.p.profile = 0;
        F.p.coarse_schedule = LTS_COARSE_FAR;   // every member's far coarse phases on the branch
        F.kc = S->kc;
        F.tsz = S->tsz;
        for (int k = 0; k < 4; ++k) F.buf[k] = E->buf[k];
        F.P1c = E->P1c;
        F.P1e = E->P1e;
        F.P2c = E->P2c;
        F.P2e = E->P2e;
        for (int k = 0; k < 3; ++k) {
            F.acc_c[k] = E->acc_c[k];
            F.acc_e[k] = E->acc_e[k];
        }
        F.q = E->q;
        F.ring_c = E->ring_c;
        F.ring_k = E->ring_k;
        F.q_side = E->q_side;
        F.ring_c_side = E->ring_c_side;
        F.ring_k_side = E->ring_k_side;
        F.flag = E->flag;
        std::vector<LaunchDesc> plan;
        make_plan(&F, parity, plan);
        F.reg = nullptr;
        const HostMesh& hm = S->reg->mesh->m;
        for (LaunchDesc& d : plan) {
            if (d.nseg == 0) continue;
            d.bytes = plan_launch_bytes(d, S->reg->r, hm.nC, hm.nE, hm.nV, S->tsz, S->kc.comp);
            for (int k = 0; k < d.nseg; ++k) {
                if (d.seg[k].elem < 0) return set_error(LTS_EINVAL, "ensembles run the three-launch path only");
                const SegDesc ps = place(E, m, d.seg[k]);
                if (ps.end > ps.begin && !placed_in_bounds(E, m, ps))
                    return set_error(LTS_EINVAL, "internal error: member %zu segment (type %d) out of bounds", m,
                                     ps.type);
                d.seg[k] = ps;
            }
        }
        plans.push_back(std::move(plan));
    }
    TablePlanStats st;
    int rc = merge_table_plan(E->kc, plans, nsm, E->arena, E->plan[parity], &st);
    if (rc != LTS_OK) return rc;
    if (parity == 0) {
        for (int k = 0; k < NKINDS; ++k) E->bytes[k] = st.bytes[k];
        E->launches = st.launches;
        E->segments = st.segments;
    }
    return LTS_OK;
}

int enqueue(lts_ensemble_s* E, const std::vector<TableLaunch>& plan, cudaStream_t st, cudaStream_t side) {
    return enqueue_table_plan(plan, E->tables, E->kc, E->flag, st, side, E->ev_fork, E->ev_join);
}

int capture(lts_ensemble_s* E) {
    for (int p = 0; p < 2; ++p) {
        cudaGraph_t g = nullptr;
        CUDA_TRY(cudaStreamBeginCapture(E->capture_stream, cudaStreamCaptureModeThreadLocal));
        int rc = enqueue(E, E->plan[p], E->capture_stream, E->capture_side);
        cudaError_t e = cudaStreamEndCapture(E->capture_stream, &g);
        if (rc != LTS_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        CUDA_TRY(e);
        e = cudaGraphInstantiate(&E->exec[p], g, 0);
        cudaGraphDestroy(g);
        CUDA_TRY(e);
    }
    return LTS_OK;
}

// Copies member m's slice of packed state vector X into (or out of) the
// member's own current state vector.
int copy_member(lts_ensemble_s* E, size_t m, bool into_member) {
    lts_state_s* S = E->members[m];
    const SV& P = E->buf[E->parity];
    const SV& X = S->buf[S->parity];
    const HostMesh& hm = S->reg->mesh->m;
    const size_t T = E->tsz;
    const size_t oc = E->offC[m] * T, oe = E->offE[m] * T;
    auto cp = [&](void* mem, void* packed, size_t off, size_t bytes) -> cudaError_t {
        if (!mem || !packed) return cudaSuccess;
        char* pk = static_cast<char*>(packed) + off;
        return into_member ? cudaMemcpyAsync(mem, pk, bytes, cudaMemcpyDeviceToDevice, E->stream)
                           : cudaMemcpyAsync(pk, mem, bytes, cudaMemcpyDeviceToDevice, E->stream);
    };
    CUDA_TRY(cp(X.hh, P.hh, oc, hm.nC * T));
    CUDA_TRY(cp(X.hl, P.hl, oc, hm.nC * T));
    CUDA_TRY(cp(X.uh, P.uh, oe, hm.nE * T));
    CUDA_TRY(cp(X.ul, P.ul, oe, hm.nE * T));
    return LTS_OK;
}

}  // namespace

namespace lts {

int merge_table_plan(const KernelConfig& kc, const std::vector<std::vector<LaunchDesc>>& plans, int nsm,
                     DeviceArena& arena, std::vector<TableLaunch>& out_plan, TablePlanStats* stats) {
    struct Group {
        LaunchDesc proto;
        std::vector<SegDesc> segs;
        double bytes = 0.0;
        bool init = false;
    };
    std::map<int, Group> groups;
    for (const auto& plan : plans)
        for (const LaunchDesc& d : plan) {
            if (d.nseg == 0) continue;   // fork / join markers are rebuilt below
            if (d.key < 0) return set_error(LTS_EINVAL, "internal error: unkeyed launch");
            Group& g = groups[d.key];
            if (!g.init) {
                g.proto = d;
                g.proto.nseg = 0;
                g.proto.fork = g.proto.join = false;
                g.init = true;
            } else if (g.proto.kind != d.kind || g.proto.in_h != d.in_h || g.proto.in_u != d.in_u ||
                       g.proto.branch != d.branch || g.proto.l2 != d.l2 || g.proto.q != d.q) {
                return set_error(LTS_EINVAL, "internal error: member plans disagree at key %d", d.key);
            }
            for (int k = 0; k < d.nseg; ++k) g.segs.push_back(d.seg[k]);
            g.bytes += d.bytes;
        }
    // device segment records of every launch, one allocation
    std::vector<std::vector<unsigned char>> recs;
    std::vector<TableLaunch> out;
    std::vector<size_t> rec_off;
    size_t total = 0;
    TablePlanStats st;
    for (auto& kv : groups) {
        Group& g = kv.second;
        TableLaunch L;
        L.d = g.proto;
        L.d.bytes = g.bytes;
        std::vector<unsigned char> rec;
        L.vblocks = encode_segment_table(kc, g.segs.data(), static_cast<int>(g.segs.size()), rec, &L.nseg);
        if (L.vblocks < 0) return set_error(LTS_EINVAL, "internal error: segment kind not tabled");
        if (L.nseg == 0) continue;
        const int per_sm = table_blocks_per_sm(kc, L.d.kind);
        L.grid = (per_sm > 0 && nsm > 0) ? per_sm * nsm : 0;
        st.bytes[L.d.kind] += g.bytes;
        st.launches += 1;
        st.segments += L.nseg;
        total = (total + 255) & ~size_t(255);
        rec_off.push_back(total);
        total += rec.size();
        recs.push_back(std::move(rec));
        out.push_back(L);
    }
    cudaError_t err = cudaSuccess;
    unsigned char* dev = static_cast<unsigned char*>(arena.alloc(std::max<size_t>(total, 256), err));
    if (err != cudaSuccess) return set_error(LTS_ENOMEM, "segment tables: %s", cudaGetErrorString(err));
    CUDA_TRY(cudaDeviceSynchronize());
    for (size_t k = 0; k < out.size(); ++k) {
        CUDA_TRY(cudaMemcpy(dev + rec_off[k], recs[k].data(), recs[k].size(), cudaMemcpyHostToDevice));
        out[k].dsegs = dev + rec_off[k];
    }
    // the concurrent branch: fork before its first launch, join before the
    // first launch of the tail, or at the end
    int first_side = -1, first_tail = -1;
    for (size_t k = 0; k < out.size(); ++k) {
        if (out[k].d.branch && first_side < 0) first_side = static_cast<int>(k);
        if (!out[k].d.branch && first_side >= 0 && first_tail < 0 &&
            k > static_cast<size_t>(first_side) && out[k].d.key >= KEY_TAIL)
            first_tail = static_cast<int>(k);
    }
    if (first_side >= 0) {
        out[first_side].d.fork = true;
        if (first_tail >= 0) {
            out[first_tail].d.join = true;
        } else {
            TableLaunch j;
            j.d.join = true;
            out.push_back(j);
        }
    }
    out_plan = std::move(out);
    if (stats) *stats = st;
    return LTS_OK;
}

int enqueue_table_plan(const std::vector<TableLaunch>& plan, const void* tables, const KernelConfig& kc,
                       int* flag, cudaStream_t st, cudaStream_t side, cudaEvent_t ev_fork, cudaEvent_t ev_join) {
    bool after_event[2] = {false, false};
    for (const auto& L : plan) {
        if (L.d.fork) {
            CUDA_TRY(cudaEventRecord(ev_fork, st));
            CUDA_TRY(cudaStreamWaitEvent(side, ev_fork, 0));
            after_event[1] = true;
        }
        if (L.d.join) {
            CUDA_TRY(cudaEventRecord(ev_join, side));
            CUDA_TRY(cudaStreamWaitEvent(st, ev_join, 0));
            after_event[0] = true;
        }
        if (L.nseg == 0) continue;
        KernelConfig k = kc;
        if (after_event[L.d.branch]) k.pdl = false;
        after_event[L.d.branch] = false;
        cudaError_t e = launch_phase_table(L.d, L.dsegs, L.nseg, L.vblocks, L.grid, tables, k, flag,
                                           L.d.branch ? side : st);
        if (e != cudaSuccess) return set_error(LTS_ECUDA, "table launch: %s", cudaGetErrorString(e));
    }
    return LTS_OK;
}

}  // namespace lts

extern "C" {

int lts_ensemble_create(const lts_state* members, int32_t n, const lts_ensemble_params* ep,
                        lts_ensemble* out) {
    if (!members || !out || n < 1) return set_error(LTS_EINVAL, "need at least one member");
    *out = nullptr;
    int rc = device_check();
    if (rc != LTS_OK) return rc;
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    std::unique_ptr<lts_ensemble_s> E(new (std::nothrow) lts_ensemble_s);
    if (!E) return set_error(LTS_ENOMEM, "out of host memory");
    const lts_state_s* s0 = members[0];
    if (!s0) return set_error(LTS_EINVAL, "null member 0");
    for (int m = 0; m < n; ++m) {
        lts_state_s* S = members[m];
        if (!S) return set_error(LTS_EINVAL, "null member %d", m);
        for (int k = 0; k < m; ++k)
            if (members[k] == S) return set_error(LTS_EINVAL, "member %d appears twice", m);
        if (S->reg->device != dev) return set_error(LTS_EINVAL, "member %d lives on another device", m);
        if (S->kc.precision != s0->kc.precision || S->kc.comp != s0->kc.comp)
            return set_error(LTS_EINVAL, "member %d: precision or compensation differs from member 0", m);
        if (S->p.mode != s0->p.mode || S->reg->r.order != s0->reg->r.order)
            return set_error(LTS_EINVAL, "member %d: mode or order differs from member 0", m);
        if (S->p.kernel_path != 0) return set_error(LTS_EINVAL, "member %d: ensembles need kernel_path 0", m);
        if (S->kc.layers != 1) return set_error(LTS_EINVAL, "member %d: ensembles take single-layer states", m);
        if (S->p.g != s0->p.g) return set_error(LTS_EINVAL, "member %d: g differs from member 0", m);
        if (S->kc.block != s0->kc.block) return set_error(LTS_EINVAL, "member %d: block size differs", m);
        E->members.push_back(S);
        E->t0.push_back(S->time);
        E->steps0.push_back(S->steps);
    }
    E->kc = s0->kc;
    E->kc.pdl = ep ? ep->pdl != 0 : true;
    E->tsz = s0->tsz;
    E->g = s0->p.g;
    // packed offsets
    E->offC.assign(n + 1, 0);
    E->offE.assign(n + 1, 0);
    E->offV.assign(n + 1, 0);
    E->oI1c.assign(n + 1, 0);
    E->oIc.assign(n + 1, 0);
    E->oI1e.assign(n + 1, 0);
    E->oIe.assign(n + 1, 0);
    int64_t tc = 0, te = 0, tv = 0;
    int maxdeg = 0, mindeg = 1 << 30, maxe_all = 0;
    for (int m = 0; m < n; ++m) {
        const HostMesh& hm = E->members[m]->reg->mesh->m;
        const RegionsHost& r = E->members[m]->reg->r;
        tc += hm.nC;
        te += hm.nE;
        tv += hm.nV;
        maxe_all = std::max(maxe_all, hm.maxE);
        if (static_cast<int64_t>(slot_rows(maxe_all)) * tc > 0x7fffffffLL || te > 0x7fffffffLL)
            return set_error(LTS_EINVAL, "ensemble too large for 32-bit indices");
        E->offC[m + 1] = static_cast<int>(tc);
        E->offE[m + 1] = static_cast<int>(te);
        E->offV[m + 1] = static_cast<int>(tv);
        E->oI1c[m + 1] = E->oI1c[m] + (r.cb[B_I1 + 1] - r.cb[B_I1]);
        E->oIc[m + 1] = E->oIc[m] + (r.cb[B_I2 + 1] - r.cb[B_I1]);
        E->oI1e[m + 1] = E->oI1e[m] + (r.eb[B_I1 + 1] - r.eb[B_I1]);
        E->oIe[m + 1] = E->oIe[m] + (r.eb[B_I2 + 1] - r.eb[B_I1]);
        E->MAXE = std::max(E->MAXE, hm.maxE);
        maxdeg = std::max(maxdeg, E->members[m]->kc.maxdeg);
        mindeg = std::min(mindeg, E->members[m]->kc.mindeg);
    }
    if (static_cast<int64_t>(E->MAXE) * tc > 0x7fffffffLL)
        return set_error(LTS_EINVAL, "ensemble too large for 32-bit indices");
    E->NC = static_cast<int>(tc);
    E->NE = static_cast<int>(te);
    E->NV = static_cast<int>(tv);
    E->kc.maxdeg = maxdeg;
    E->kc.mindeg = mindeg;
    rc = E->kc.precision ? build_union_tables<double>(E.get(), E->t64) : build_union_tables<float>(E.get(), E->t32);
    if (rc != LTS_OK) return rc;
    E->tables = E->kc.precision ? static_cast<const void*>(&E->t64) : static_cast<const void*>(&E->t32);
    rc = alloc_state(E.get());
    if (rc != LTS_OK) return rc;
    int nsm = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    if (!ep || !ep->persistent) nsm = 0;   // one block per virtual block (the default)
    for (int p = 0; p < 2; ++p) {
        rc = build_plan(E.get(), p, nsm);
        if (rc != LTS_OK) return rc;
    }
    if (ep && ep->stream) {
        E->stream = static_cast<cudaStream_t>(ep->stream);
    } else {
        CUDA_TRY(cudaStreamCreateWithFlags(&E->stream, cudaStreamNonBlocking));
        E->own_stream = true;
    }
    CUDA_TRY(cudaStreamCreateWithFlags(&E->capture_stream, cudaStreamNonBlocking));
    CUDA_TRY(cudaStreamCreateWithFlags(&E->capture_side, cudaStreamNonBlocking));
    CUDA_TRY(cudaStreamCreateWithFlags(&E->side_stream, cudaStreamNonBlocking));
    CUDA_TRY(cudaEventCreateWithFlags(&E->ev_fork, cudaEventDisableTiming));
    CUDA_TRY(cudaEventCreateWithFlags(&E->ev_join, cudaEventDisableTiming));
    CUDA_TRY(cudaEventCreateWithFlags(&E->ev_io, cudaEventDisableTiming));
    CUDA_TRY(cudaHostAlloc(reinterpret_cast<void**>(&E->flag_host), sizeof(int), cudaHostAllocDefault));
    // the members' current states become the packed state
    for (int m = 0; m < n; ++m) CUDA_TRY(cudaStreamSynchronize(E->members[m]->stream));
    for (int m = 0; m < n; ++m) {
        rc = copy_member(E.get(), m, false);
        if (rc != LTS_OK) return rc;
    }
    if (!ep || ep->use_graph) {
        rc = capture(E.get());
        if (rc != LTS_OK) return rc;
    }
    CUDA_TRY(cudaStreamSynchronize(E->stream));
    *out = E.release();
    return LTS_OK;
}

void lts_ensemble_destroy(lts_ensemble e) {
    if (!e) return;
    cudaStreamSynchronize(e->stream);
    delete e;
}

int lts_ensemble_step(lts_ensemble e, int32_t n) {
    if (!e) return set_error(LTS_EINVAL, "null ensemble");
    if (n < 0) return set_error(LTS_EINVAL, "n_coarse must be >= 0");
    for (int i = 0; i < n; ++i) {
        if (e->exec[e->parity]) {
            CUDA_TRY(cudaGraphLaunch(e->exec[e->parity], e->stream));
        } else {
            int rc = enqueue(e, e->plan[e->parity], e->stream, e->side_stream);
            if (rc != LTS_OK) return rc;
        }
        e->parity ^= 1;
        e->steps++;
    }
    return LTS_OK;
}

int lts_ensemble_read(lts_ensemble e, int32_t i, double* h, double* u, lts_diag* d) {
    if (!e) return set_error(LTS_EINVAL, "null ensemble");
    if (i < 0 || i >= static_cast<int32_t>(e->members.size()))
        return set_error(LTS_EINVAL, "member index %d out of range", i);
    lts_state_s* S = e->members[i];
    // unpack only after the member's previous gathers (an asynchronous read)
    CUDA_TRY(cudaStreamWaitEvent(e->stream, S->ev_out_u, 0));
    int rc = copy_member(e, i, true);
    if (rc != LTS_OK) return rc;
    // the flag copy and the unpacking happen on the ensemble's stream; the
    // member's read waits for them there and synchronises its own streams
    CUDA_TRY(cudaMemcpyAsync(e->flag_host, e->flag, sizeof(int), cudaMemcpyDeviceToHost, e->stream));
    CUDA_TRY(cudaMemsetAsync(e->flag, 0, sizeof(int), e->stream));
    CUDA_TRY(cudaEventRecord(e->ev_io, e->stream));
    CUDA_TRY(cudaStreamWaitEvent(S->stream, e->ev_io, 0));
    S->steps = e->steps0[i] + e->steps;
    S->time = e->t0[i] + static_cast<double>(e->steps) * S->p.dt;
    rc = lts_read(S, h, u, d);
    if (rc != LTS_OK) return rc;
    const int flag = *e->flag_host;
    if (flag & 4) return set_error(LTS_ECUDA, "internal error: a tile exceeded its shared memory (skipped)");
    if (flag)
        return set_error(LTS_ENONFINITE, "an ensemble stage produced %s",
                         (flag & 1) ? "a thickness <= 0 or non-finite" : "a non-finite velocity");
    return LTS_OK;
}

int lts_ensemble_read_async(lts_ensemble e, int32_t i, double* h, double* u, lts_diag* d) {
    if (!e) return set_error(LTS_EINVAL, "null ensemble");
    if (i < 0 || i >= static_cast<int32_t>(e->members.size()))
        return set_error(LTS_EINVAL, "member index %d out of range", i);
    lts_state_s* S = e->members[i];
    CUDA_TRY(cudaStreamWaitEvent(e->stream, S->ev_out_u, 0));
    int rc = copy_member(e, i, true);
    if (rc != LTS_OK) return rc;
    CUDA_TRY(cudaEventRecord(e->ev_io, e->stream));
    CUDA_TRY(cudaStreamWaitEvent(S->stream, e->ev_io, 0));
    S->steps = e->steps0[i] + e->steps;
    S->time = e->t0[i] + static_cast<double>(e->steps) * S->p.dt;
    return lts_read_async(S, h, u, d);
}

int lts_ensemble_sync(lts_ensemble e) {
    if (!e) return set_error(LTS_EINVAL, "null ensemble");
    CUDA_TRY(cudaMemcpyAsync(e->flag_host, e->flag, sizeof(int), cudaMemcpyDeviceToHost, e->stream));
    CUDA_TRY(cudaMemsetAsync(e->flag, 0, sizeof(int), e->stream));
    CUDA_TRY(cudaStreamSynchronize(e->stream));
    int rc = LTS_OK;
    for (lts_state_s* S : e->members) {
        const int r = lts_sync(S);
        if (r != LTS_OK && rc == LTS_OK) rc = r;
    }
    if (rc != LTS_OK) return rc;
    const int flag = *e->flag_host;
    if (flag & 4) return set_error(LTS_ECUDA, "internal error: a tile exceeded its shared memory (skipped)");
    if (flag)
        return set_error(LTS_ENONFINITE, "an ensemble stage produced %s",
                         (flag & 1) ? "a thickness <= 0 or non-finite" : "a non-finite velocity");
    return LTS_OK;
}

int lts_ensemble_write(lts_ensemble e, int32_t i, const double* h, const double* u, double time,
                       int64_t steps) {
    if (!e || !h || !u) return set_error(LTS_EINVAL, "null argument");
    if (i < 0 || i >= static_cast<int32_t>(e->members.size()))
        return set_error(LTS_EINVAL, "member index %d out of range", i);
    lts_state_s* S = e->members[i];
    int rc = lts_write(S, h, u, time, steps);
    if (rc != LTS_OK) return rc;
    // packing waits for the member's scatter on the ensemble's stream
    CUDA_TRY(cudaEventRecord(e->ev_io, S->stream));
    CUDA_TRY(cudaStreamWaitEvent(e->stream, e->ev_io, 0));
    rc = copy_member(e, i, false);
    if (rc != LTS_OK) return rc;
    // the member's clock restarts here; later reads add the ensemble's steps
    e->t0[i] = time - static_cast<double>(e->steps) * S->p.dt;
    e->steps0[i] = steps - e->steps;
    return LTS_OK;
}

int lts_ensemble_stats(lts_ensemble e, int32_t* launches_per_step, double* bytes, int64_t* cells,
                       int32_t* segments_per_step) {
    if (!e) return set_error(LTS_EINVAL, "null ensemble");
    if (launches_per_step) *launches_per_step = e->launches;
    if (bytes)
        for (int k = 0; k < NKINDS; ++k) bytes[k] = e->bytes[k];
    if (cells) *cells = e->NC;
    if (segments_per_step) *segments_per_step = e->segments;
    return LTS_OK;
}

}  // extern "C"
