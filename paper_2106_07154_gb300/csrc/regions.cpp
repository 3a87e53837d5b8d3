// regions.cpp -- region labelling of Eqs. (3)-(5), band ordering and the
// band-ordered kernel tables (host side of liblts.so).
//
// Labelling: breadth-first edge distances from the fine set F (outwards) and
// from the non-fine cells (into F).  With L cells per interface layer:
//   I1 = non-F cells at distance 1..L, I2 = distance L+1..2L   (Eq. 3)
//   F1 = F cells at inner distance 1, F2 = inner distance 2    (Eq. 4)
// and every edge takes the finer of its two cells' regions, i.e. edges are
// assigned from the fine to the coarse side (Eq. 5).
// Bands (order of the device arrays):
//   0 F deep | 1 F3 | 2 F2 | 3 F1 | 4 I1 | 5 I2 | 6..10 C1..C5 | 11 C rest
// F3 is the fine layer next to F2, C1..C5 the coarse layers next to I2
// (the halo layers the restricted right-hand sides read).  Cells are in
// Hilbert-curve order inside a band, edges follow their lower-indexed cell,
// vertices their lowest cell.  Adjacent cells differ by at most one band, so
// a right-hand side updating bands [lo, hi] reads bands [lo-1, hi+2] only.
#include "regions.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "lts_error.h"

namespace lts {

namespace {

// Hilbert index of a point of the unit cube (Skilling, "Programming the
// Hilbert curve", AIP Conf. Proc. 707, 2004): axes -> transposed form, then
// the bits are interleaved.
uint64_t hilbert3(double x, double y, double z) {
    const int b = 21;
    auto q = [](double v) {
        v = std::min(std::max(v, 0.0), 1.0);
        return static_cast<uint32_t>(v * ((1u << 21) - 1));
    };
    uint32_t X[3] = {q(x), q(y), q(z)};
    const uint32_t M = 1u << (b - 1);
    for (uint32_t Q = M; Q > 1; Q >>= 1) {
        uint32_t P = Q - 1;
        for (int i = 0; i < 3; ++i) {
            if (X[i] & Q) {
                X[0] ^= P;
            } else {
                uint32_t t = (X[0] ^ X[i]) & P;
                X[0] ^= t;
                X[i] ^= t;
            }
        }
    }
    for (int i = 1; i < 3; ++i) X[i] ^= X[i - 1];
    uint32_t t = 0;
    for (uint32_t Q = M; Q > 1; Q >>= 1)
        if (X[2] & Q) t ^= Q - 1;
    for (int i = 0; i < 3; ++i) X[i] ^= t;
    uint64_t key = 0;
    for (int bit = b - 1; bit >= 0; --bit)
        for (int i = 0; i < 3; ++i) key = (key << 1) | ((X[i] >> bit) & 1u);
    return key;
}

std::vector<int> bfs(const HostMesh& m, const std::vector<char>& source,
                     const std::vector<char>& allowed) {
    const int INF = 1 << 30;
    std::vector<int> d(m.nC, INF), frontier, next;
    for (int i = 0; i < m.nC; ++i)
        if (source[i]) {
            d[i] = 0;
            frontier.push_back(i);
        }
    while (!frontier.empty()) {
        next.clear();
        for (int i : frontier)
            for (int j = 0; j < m.nEoC[i]; ++j) {
                int nb = m.CoC[static_cast<size_t>(i) * m.maxE + j];
                if (allowed[nb] && d[nb] == INF) {
                    d[nb] = d[i] + 1;
                    next.push_back(nb);
                }
            }
        frontier.swap(next);
    }
    return d;
}

}  // namespace

namespace {
int regions_impl(const HostMesh& m, const int8_t* fine, int layers, int ordering, RegionsHost& r,
                 const int8_t* rid, int nreg);
}

int compute_regions(const HostMesh& m, const int8_t* fine, int layers, int ordering, RegionsHost& r) {
    return regions_impl(m, fine, layers, ordering, r, nullptr, 1);
}

int compute_regions_multi(const HostMesh& m, const int8_t* region_of_cell, int nreg, int layers, int ordering,
                          RegionsHost& r) {
    if (nreg < 1 || nreg > 64) return set_error(LTS_EINVAL, "number of regions must be in [1, 64]");
    std::vector<int8_t> fine(m.nC);
    for (int i = 0; i < m.nC; ++i) {
        if (region_of_cell[i] < 0 || region_of_cell[i] > nreg)
            return set_error(LTS_EINVAL, "region id %d of cell %d out of range", region_of_cell[i], i);
        fine[i] = region_of_cell[i] > 0;
    }
    const int rc = regions_impl(m, fine.data(), layers, ordering, r, nreg > 1 ? region_of_cell : nullptr, nreg);
    if (rc == LTS_OK) r.rid.assign(region_of_cell, region_of_cell + m.nC);
    return rc;
}

namespace {
int regions_impl(const HostMesh& m, const int8_t* fine, int layers, int ordering, RegionsHost& r,
                 const int8_t* rid, int nreg) {
    if (layers < 1) return set_error(LTS_EINVAL, "interface_layers must be >= 1");
    if (ordering != 0 && ordering != 1) return set_error(LTS_EINVAL, "ordering must be 0 or 1");
    r.ordering = ordering;
    r.fine.assign(fine, fine + m.nC);
    const int nC = m.nC, nE = m.nE, nV = m.nV;
    std::vector<char> isF(nC), notF(nC), all(nC, 1);
    for (int i = 0; i < nC; ++i) {
        isF[i] = fine[i] != 0;
        notF[i] = !isF[i];
    }
    std::vector<int> dout = bfs(m, isF, all);   // distance from F
    std::vector<int> din = bfs(m, notF, all);   // distance from the non-fine cells
    r.layers = layers;
    r.cband.assign(nC, B_CREST);
    for (int i = 0; i < nC; ++i) {
        int b;
        if (isF[i]) {
            int d = din[i];
            b = d == 1 ? B_F1 : d == 2 ? B_F2 : d == 3 ? B_F3 : B_FDEEP;
        } else {
            int d = dout[i];
            if (d <= layers) b = B_I1;
            else if (d <= 2 * layers) b = B_I2;
            else if (d - 2 * layers <= 5) b = B_C1 + (d - 2 * layers - 1);   // C1..C5
            else b = B_CREST;
        }
        r.cband[i] = static_cast<int8_t>(b);
    }
    r.eband.assign(nE, 0);
    for (int e = 0; e < nE; ++e)
        r.eband[e] = std::min(r.cband[m.CoE[2 * e]], r.cband[m.CoE[2 * e + 1]]);
    r.vband.assign(nV, 0);
    for (int v = 0; v < nV; ++v)
        r.vband[v] = std::min({r.cband[m.CoV[3 * v]], r.cband[m.CoV[3 * v + 1]], r.cband[m.CoV[3 * v + 2]]});

    // ---- blocks: one region's near bands (F deep..C5) per block, then the far
    //      coarse cells; a single region is block 0 and C rest block 1
    r.nreg = nreg;
    std::vector<int> cblock(nC, 0);
    if (!rid) {
        for (int i = 0; i < nC; ++i) cblock[i] = r.cband[i] == B_CREST ? 1 : 0;
    } else {
        // walk out of each region's fine cells through the near bands; the
        // bands up to C2 (which Step 3 reads) must not meet another region's
        std::vector<int> reg(nC, 0), queue;
        queue.reserve(nC);
        for (int i = 0; i < nC; ++i)
            if (fine[i]) {
                reg[i] = rid[i];
                queue.push_back(i);
            }
        for (size_t h = 0; h < queue.size(); ++h) {
            const int i = queue[h];
            for (int j = 0; j < m.nEoC[i]; ++j) {
                const int nb = m.CoC[static_cast<size_t>(i) * m.maxE + j];
                if (r.cband[nb] == B_CREST) continue;
                if (reg[nb] == 0) {
                    reg[nb] = reg[i];
                    queue.push_back(nb);
                } else if (reg[nb] != reg[i] && r.cband[nb] <= B_C2 && r.cband[i] <= B_C2) {
                    return set_error(LTS_EINVAL,
                                     "fine regions %d and %d are too close: their fine, interface and first "
                                     "two coarse layers touch", reg[i], reg[nb]);
                }
            }
        }
        for (int i = 0; i < nC; ++i) cblock[i] = r.cband[i] == B_CREST ? nreg : reg[i] - 1;
    }
    auto eblock = [&](int e) {
        const int a = m.CoE[2 * e], b = m.CoE[2 * e + 1];
        return r.cband[a] <= r.cband[b] ? cblock[a] : cblock[b];
    };
    auto vblock = [&](int v) {
        int best = m.CoV[3 * v];
        for (int q = 1; q < 3; ++q)
            if (r.cband[m.CoV[3 * v + q]] < r.cband[best]) best = m.CoV[3 * v + q];
        return cblock[best];
    };
    // ---- cells: block, band, then Hilbert key (or the mesh's own index)
    std::vector<uint64_t> key(nC);
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int i = 0; i < nC; ++i) {
        double p[3] = {m.xc[i], m.yc[i], m.zc[i]};
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::min(lo[k], p[k]);
            hi[k] = std::max(hi[k], p[k]);
        }
    }
    for (int i = 0; i < nC; ++i) {
        double p[3] = {m.xc[i], m.yc[i], m.zc[i]};
        double s[3];
        for (int k = 0; k < 3; ++k) s[k] = hi[k] > lo[k] ? (p[k] - lo[k]) / (hi[k] - lo[k]) : 0.0;
        key[i] = ordering == 0 ? hilbert3(s[0], s[1], s[2]) : static_cast<uint64_t>(i);
    }
    r.perm_c.resize(nC);
    std::iota(r.perm_c.begin(), r.perm_c.end(), 0);
    std::stable_sort(r.perm_c.begin(), r.perm_c.end(), [&](int a, int b) {
        if (cblock[a] != cblock[b]) return cblock[a] < cblock[b];
        if (r.cband[a] != r.cband[b]) return r.cband[a] < r.cband[b];
        return key[a] < key[b];
    });
    r.inv_c.resize(nC);
    for (int k = 0; k < nC; ++k) r.inv_c[r.perm_c[k]] = k;
    // ---- edges: band, then their lower new cell index
    r.perm_e.resize(nE);
    std::iota(r.perm_e.begin(), r.perm_e.end(), 0);
    auto ekey = [&](int e) {
        int a = r.inv_c[m.CoE[2 * e]], b = r.inv_c[m.CoE[2 * e + 1]];
        return std::make_pair(std::min(a, b), std::max(a, b));
    };
    std::vector<int> eblk(nE);
    for (int e = 0; e < nE; ++e) eblk[e] = eblock(e);
    std::stable_sort(r.perm_e.begin(), r.perm_e.end(), [&](int a, int b) {
        if (eblk[a] != eblk[b]) return eblk[a] < eblk[b];
        if (r.eband[a] != r.eband[b]) return r.eband[a] < r.eband[b];
        return ekey(a) < ekey(b);
    });
    r.inv_e.resize(nE);
    for (int k = 0; k < nE; ++k) r.inv_e[r.perm_e[k]] = k;
    // ---- vertices: band, then their lowest new cell index
    r.perm_v.resize(nV);
    std::iota(r.perm_v.begin(), r.perm_v.end(), 0);
    auto vkey = [&](int v) {
        int a = r.inv_c[m.CoV[3 * v]], b = r.inv_c[m.CoV[3 * v + 1]], c = r.inv_c[m.CoV[3 * v + 2]];
        return std::min({a, b, c});
    };
    std::vector<int> vblk(nV);
    for (int v = 0; v < nV; ++v) vblk[v] = vblock(v);
    std::stable_sort(r.perm_v.begin(), r.perm_v.end(), [&](int a, int b) {
        if (vblk[a] != vblk[b]) return vblk[a] < vblk[b];
        if (r.vband[a] != r.vband[b]) return r.vband[a] < r.vband[b];
        return vkey(a) < vkey(b);
    });
    r.inv_v.resize(nV);
    for (int k = 0; k < nV; ++k) r.inv_v[r.perm_v[k]] = k;
    // ---- band offsets
    for (int k = 0; k <= NBANDS; ++k) r.cb[k] = r.eb[k] = r.vb[k] = 0;
    for (int i = 0; i < nC; ++i) r.cb[r.cband[i] + 1]++;
    for (int e = 0; e < nE; ++e) r.eb[r.eband[e] + 1]++;
    for (int v = 0; v < nV; ++v) r.vb[r.vband[v] + 1]++;
    for (int k = 0; k < NBANDS; ++k) {
        r.cb[k + 1] += r.cb[k];
        r.eb[k + 1] += r.eb[k];
        r.vb[k + 1] += r.vb[k];
    }
    // ---- band offsets of every block as the planner of that block sees them
    //      (several regions only; a single region uses cb, eb, vb)
    r.mcb.clear();
    r.meb.clear();
    r.mvb.clear();
    if (rid) {
        const int nb = nreg + 1;
        auto offsets = [&](const std::vector<int8_t>& band, const std::vector<int>& blk, int n,
                           std::vector<std::vector<int>>& out) {
            // count[b][k], then prefix in (block, band) order
            std::vector<std::vector<int>> cnt(nb, std::vector<int>(NBANDS, 0));
            for (int x = 0; x < n; ++x) cnt[blk[x]][band[x]]++;
            out.assign(nb, std::vector<int>(NBANDS + 1, 0));
            int pos = 0;
            for (int b = 0; b < nb; ++b) {
                for (int k = 0; k < NBANDS; ++k) {
                    out[b][k] = pos;
                    pos += cnt[b][k];
                }
                out[b][NBANDS] = pos;
            }
        };
        offsets(r.cband, cblock, nC, r.mcb);
        offsets(r.eband, eblk, nE, r.meb);
        offsets(r.vband, vblk, nV, r.mvb);
    }
    // ---- connectivity in band order (host copies, for the planner's byte counts)
    const int W = m.maxE, WR = slot_rows(W);
    r.cn.assign(nC, 0);
    r.se.assign(static_cast<size_t>(WR) * nC, 0);
    r.sn.assign(static_cast<size_t>(WR) * nC, 0);
    r.sv.assign(static_cast<size_t>(WR) * nC, 0);
    for (int k = 0; k < nC; ++k) {
        int c = r.perm_c[k];
        int n = m.nEoC[c];
        r.cn[k] = static_cast<uint8_t>(n);
        for (int j = 0; j < WR; ++j) {
            int jj = j < n ? j : 0;     // padding slots repeat slot 0 (never read)
            r.se[static_cast<size_t>(j) * nC + k] = r.inv_e[m.EoC[static_cast<size_t>(c) * W + jj]];
            r.sn[static_cast<size_t>(j) * nC + k] = r.inv_c[m.CoC[static_cast<size_t>(c) * W + jj]];
            r.sv[static_cast<size_t>(j) * nC + k] = r.inv_v[m.VoC[static_cast<size_t>(c) * W + jj]];
        }
    }
    r.ec0.resize(nE);
    r.ec1.resize(nE);
    r.ep.resize(nE);
    for (int k = 0; k < nE; ++k) {
        int e = r.perm_e[k];
        int c0 = m.CoE[2 * e], c1 = m.CoE[2 * e + 1];
        r.ec0[k] = r.inv_c[c0];
        r.ec1[k] = r.inv_c[c1];
        int p0 = -1, p1 = -1;
        for (int j = 0; j < m.nEoC[c0]; ++j)
            if (m.EoC[static_cast<size_t>(c0) * W + j] == e) p0 = j;
        for (int j = 0; j < m.nEoC[c1]; ++j)
            if (m.EoC[static_cast<size_t>(c1) * W + j] == e) p1 = j;
        if (p0 < 0 || p1 < 0) return set_error(LTS_EINVAL, "edge %d missing from its cells' rings", e);
        r.ep[k] = static_cast<uint32_t>(p0) | (static_cast<uint32_t>(p1) << 8);
    }
    r.vc.assign(3 * static_cast<size_t>(nV), 0);
    r.ve.assign(3 * static_cast<size_t>(nV), 0);
    (void)0;
    for (int k = 0; k < nV; ++k) {
        int v = r.perm_v[k];
        for (int q = 0; q < 3; ++q) {
            r.vc[static_cast<size_t>(q) * nV + k] = r.inv_c[m.CoV[3 * v + q]];
            r.ve[static_cast<size_t>(q) * nV + k] = r.inv_e[m.EoV[3 * v + q]];
        }
    }
    return LTS_OK;
}
}  // namespace


// Tiles for the fused right-hand-side kernel.  Tile cells are a contiguous
// band-order range inside one band; the tile owns the edges whose lower
// band-order cell is one of its cells (edges are sorted by that cell, so this
// is an edge range, and all such edges carry the tile's band).  The tile's
// local cells are its own cells followed by its halo (the other cell of owned
// edges); its local vertices are all ring vertices of its local cells.
int build_tiles(const HostMesh& m, RegionsHost& r, int tile_cells) {
    const int nC = m.nC, nE = m.nE, WR = slot_rows(m.maxE);
    if (tile_cells < 32 || tile_cells > 4096) return set_error(LTS_EINVAL, "tile size out of range");
    r.tile_cells = tile_cells;
    r.tile_a.clear();
    r.tile_b.clear();
    r.tile_lsv_off.clear();
    r.halo.clear();
    r.tverts.clear();
    r.lsv.clear();
    r.lec.assign(nE, 0);
    r.max_local_cells = r.max_local_verts = 0;
    // edges are sorted by (band, lower cell): lower cell of every edge
    std::vector<int> lowc(nE);
    for (int e = 0; e < nE; ++e) lowc[e] = std::min(r.ec0[e], r.ec1[e]);
    std::vector<int> stamp_c(nC, -1), local_c(nC, -1), stamp_v(m.nV, -1), local_v(m.nV, -1);
    int ecur = 0;
    for (int b = 0; b < NBANDS; ++b) {
        r.tb[b] = static_cast<int>(r.tile_a.size());
        for (int c0 = r.cb[b]; c0 < r.cb[b + 1]; c0 += tile_cells) {
            const int c1 = std::min(c0 + tile_cells, r.cb[b + 1]);
            const int t = static_cast<int>(r.tile_a.size());
            // owned edges: lower cell in [c0, c1)
            while (ecur < nE && lowc[ecur] < c0) ++ecur;
            const int e0 = ecur;
            while (ecur < nE && lowc[ecur] < c1) ++ecur;
            const int e1 = ecur;
            // local cells: own cells, then halo
            std::vector<int> cells;
            for (int c = c0; c < c1; ++c) {
                stamp_c[c] = t;
                local_c[c] = static_cast<int>(cells.size());
                cells.push_back(c);
            }
            const int halo_begin = static_cast<int>(r.halo.size());
            for (int e = e0; e < e1; ++e) {
                for (int c : {r.ec0[e], r.ec1[e]}) {
                    if (stamp_c[c] != t) {
                        stamp_c[c] = t;
                        local_c[c] = static_cast<int>(cells.size());
                        cells.push_back(c);
                        r.halo.push_back(c);
                    }
                }
                r.lec[e] = static_cast<uint32_t>(local_c[r.ec0[e]]) |
                           (static_cast<uint32_t>(local_c[r.ec1[e]]) << 16);
            }
            const int nl = static_cast<int>(cells.size());
            // local vertices: ring vertices of the local cells, first seen first
            const int vert_begin = static_cast<int>(r.tverts.size());
            int nv = 0;
            for (int c : cells)
                for (int j = 0; j < r.cn[c]; ++j) {
                    int v = r.sv[static_cast<size_t>(j) * nC + c];
                    if (stamp_v[v] != t) {
                        stamp_v[v] = t;
                        local_v[v] = nv++;
                        r.tverts.push_back(v);
                    }
                }
            if (nl > 65535 || nv > 65535) return set_error(LTS_EINVAL, "tile too large");
            // lsv block, slot-major over the local cells
            r.tile_lsv_off.push_back(static_cast<int>(r.lsv.size()));
            const size_t base = r.lsv.size();
            r.lsv.resize(base + static_cast<size_t>(WR) * nl, 0);
            for (int k = 0; k < nl; ++k) {
                int c = cells[k];
                for (int j = 0; j < r.cn[c]; ++j)
                    r.lsv[base + static_cast<size_t>(j) * nl + k] =
                        static_cast<uint16_t>(local_v[r.sv[static_cast<size_t>(j) * nC + c]]);
            }
            r.tile_a.push_back(make_int4(c0, c1 - c0, halo_begin, nl));
            r.tile_b.push_back(make_int4(e0, e1, vert_begin, nv));
            r.max_local_cells = std::max(r.max_local_cells, nl);
            r.max_local_verts = std::max(r.max_local_verts, nv);
        }
    }
    r.tb[NBANDS] = static_cast<int>(r.tile_a.size());
    r.ntiles = r.tb[NBANDS];
    if (ecur != nE) return set_error(LTS_EINVAL, "tiles do not cover the edges");
    return LTS_OK;
}

// Coefficient tables, derived in FP64 from the master geometry and rounded
// once to T.
template <class T>
void coefficient_tables(const HostMesh& m, const RegionsHost& r, CoefTables<T>& o) {
    const int nC = m.nC, nE = m.nE, nV = m.nV, W = m.maxE, WR = slot_rows(W);
    o.snl.assign(static_cast<size_t>(WR) * nC, T(0));
    o.sR.assign(static_cast<size_t>(WR) * nC, T(0));
    o.sK.assign(static_cast<size_t>(WR) * nC, T(0));
    o.sK64.assign(static_cast<size_t>(WR) * nC, 0.0);
    o.rA.resize(nC);
    o.b.resize(nC);
    o.area.resize(nC);
    o.bd.resize(nC);
    for (int k = 0; k < nC; ++k) {
        int c = r.perm_c[k];
        int n = m.nEoC[c];
        double A = m.A[c];
        for (int j = 0; j < n; ++j) {
            int e = m.EoC[static_cast<size_t>(c) * W + j];
            int v = m.VoC[static_cast<size_t>(c) * W + j];
            double nsign = (m.CoE[2 * e] == c) ? 1.0 : -1.0;
            double kite = 0.0;
            for (int q = 0; q < 3; ++q)
                if (m.CoV[3 * v + q] == c) kite = m.kite[3 * v + q];
            size_t at = static_cast<size_t>(j) * nC + k;
            o.snl[at] = static_cast<T>(nsign * m.dv[e]);
            o.sR[at] = static_cast<T>(kite / A);
            double kc = m.dv[e] * m.dc[e] / (4.0 * A);
            o.sK[at] = static_cast<T>(kc);
            o.sK64[at] = kc;
        }
        o.rA[k] = static_cast<T>(1.0 / A);
        o.b[k] = static_cast<T>(m.b[c]);
        o.area[k] = A;
        o.bd[k] = m.b[c];
    }
    o.rdc.resize(nE);
    for (int k = 0; k < nE; ++k) o.rdc[k] = static_cast<T>(1.0 / m.dc[r.perm_e[k]]);
    // the bottom difference across each edge, subtracted in T exactly as a
    // kernel would subtract the two cells' T values (so the edge pass needs
    // no dependent gather of b)
    o.db.resize(nE);
    for (int k = 0; k < nE; ++k) {
        const T b1 = o.b[r.ec1[k]], b0 = o.b[r.ec0[k]];
        o.db[k] = b1 - b0;
    }
    o.vk.assign(3 * static_cast<size_t>(nV), T(0));
    o.vd.assign(3 * static_cast<size_t>(nV), T(0));
    o.f.resize(nV);
    for (int k = 0; k < nV; ++k) {
        int v = r.perm_v[k];
        double Av = m.Av[v];
        for (int q = 0; q < 3; ++q) {
            int e = m.EoV[3 * v + q];
            double t = (m.VoE[2 * e + 1] == v) ? 1.0 : -1.0;
            o.vk[static_cast<size_t>(q) * nV + k] = static_cast<T>(m.kite[3 * v + q] / Av);
            o.vd[static_cast<size_t>(q) * nV + k] = static_cast<T>(t * m.dc[e] / Av);
        }
        o.f[k] = static_cast<T>(m.f[v]);
    }
}

template void coefficient_tables<float>(const HostMesh&, const RegionsHost&, CoefTables<float>&);
template void coefficient_tables<double>(const HostMesh&, const RegionsHost&, CoefTables<double>&);

template <class T>
void pack_ring_slots(const std::vector<int>& se, const std::vector<int>& sn, const std::vector<int>& sv,
                     const std::vector<T>& snl, const std::vector<T>& sR, const std::vector<T>& sK,
                     std::vector<int4>& sidx, std::vector<float2>& scf) {
    const size_t n = se.size();
    sidx.resize(n);
    scf.assign(sizeof(T) == 4 ? n : 0, float2{});
    for (size_t x = 0; x < n; ++x) {
        int bits = 0;
        if (sizeof(T) == 4) {
            const float f = static_cast<float>(snl[x]);
            std::memcpy(&bits, &f, sizeof(bits));
            scf[x].x = static_cast<float>(sR[x]);
            scf[x].y = static_cast<float>(sK[x]);
        }
        sidx[x].x = se[x];
        sidx[x].y = sn[x];
        sidx[x].z = sv[x];
        sidx[x].w = bits;
    }
}
template void pack_ring_slots<float>(const std::vector<int>&, const std::vector<int>&, const std::vector<int>&,
                                     const std::vector<float>&, const std::vector<float>&,
                                     const std::vector<float>&, std::vector<int4>&, std::vector<float2>&);
template void pack_ring_slots<double>(const std::vector<int>&, const std::vector<int>&, const std::vector<int>&,
                                      const std::vector<double>&, const std::vector<double>&,
                                      const std::vector<double>&, std::vector<int4>&, std::vector<float2>&);

template <class T>
void pack_edge_vertex_rows(const std::vector<int>& ec0, const std::vector<int>& ec1,
                           const std::vector<uint32_t>& ep, const std::vector<T>& rdc, const std::vector<int>& vc,
                           const std::vector<int>& ve, const std::vector<T>& vd, const std::vector<T>& vk,
                           const std::vector<T>& f, std::vector<int4>& erow, std::vector<int4>& vri,
                           std::vector<float4>& vrd, std::vector<float4>& vrk) {
    const bool fp32 = sizeof(T) == 4;
    auto bits = [](T x) {
        const float y = static_cast<float>(x);
        int b = 0;
        std::memcpy(&b, &y, sizeof(b));
        return b;
    };
    auto as_float = [](int x) {
        float y = 0.f;
        std::memcpy(&y, &x, sizeof(y));
        return y;
    };
    const size_t nE = ec0.size(), nV = f.size();
    erow.resize(nE);
    for (size_t e = 0; e < nE; ++e)
        erow[e] = int4{ec0[e], ec1[e], static_cast<int>(ep[e]), fp32 ? bits(rdc[e]) : 0};
    vri.resize(nV);
    vrd.assign(fp32 ? nV : 0, float4{});
    vrk.assign(fp32 ? nV : 0, float4{});
    for (size_t v = 0; v < nV; ++v) {
        vri[v] = int4{ve[v], ve[nV + v], ve[2 * nV + v], vc[v]};
        if (fp32) {
            vrd[v] = float4{static_cast<float>(vd[v]), static_cast<float>(vd[nV + v]),
                            static_cast<float>(vd[2 * nV + v]), static_cast<float>(f[v])};
            vrk[v] = float4{static_cast<float>(vk[v]), static_cast<float>(vk[nV + v]),
                            static_cast<float>(vk[2 * nV + v]), as_float(vc[nV + v])};
        }
    }
}
template void pack_edge_vertex_rows<float>(const std::vector<int>&, const std::vector<int>&,
                                           const std::vector<uint32_t>&, const std::vector<float>&,
                                           const std::vector<int>&, const std::vector<int>&,
                                           const std::vector<float>&, const std::vector<float>&,
                                           const std::vector<float>&, std::vector<int4>&, std::vector<int4>&,
                                           std::vector<float4>&, std::vector<float4>&);
template void pack_edge_vertex_rows<double>(const std::vector<int>&, const std::vector<int>&,
                                            const std::vector<uint32_t>&, const std::vector<double>&,
                                            const std::vector<int>&, const std::vector<int>&,
                                            const std::vector<double>&, const std::vector<double>&,
                                            const std::vector<double>&, std::vector<int4>&, std::vector<int4>&,
                                            std::vector<float4>&, std::vector<float4>&);

// TRiSK weight of Eq. (weights) for e' = slot j of cell c and e = slot p,
// with the path taken counter-clockwise from e' to e (used to validate a
// caller's weightsOnEdge).
double derived_weight(const HostMesh& m, int c, int j, int p) {
    const int W = m.maxE;
    const int n = m.nEoC[c];
    double S = 0.0;
    for (int q = j; q != p; q = (q + 1) % n) {
        int v = m.VoC[static_cast<size_t>(c) * W + q];
        for (int s = 0; s < 3; ++s)
            if (m.CoV[3 * v + s] == c) S += m.kite[3 * v + s] / m.A[c];
    }
    int ep = m.EoC[static_cast<size_t>(c) * W + j];
    int e = m.EoC[static_cast<size_t>(c) * W + p];
    double n_ep = (m.CoE[2 * ep] == c) ? 1.0 : -1.0;
    double n_e = (m.CoE[2 * e] == c) ? 1.0 : -1.0;
    return n_ep * (-n_e) * (S - 0.5);
}

}  // namespace lts
