// regions.h -- host-side mesh copy, region labels and band ordering.
#pragma once
#include <cstdint>
#include <vector>

#include "../../include/lts.h"
#include "lts_internal.h"

namespace lts {

// Validated copy of an lts_mesh_desc (original index order, FP64 master).
struct HostMesh {
    int nC = 0, nE = 0, nV = 0, maxE = 0;
    bool sphere = false;
    double R = 0, Lx = 0, Ly = 0;
    std::vector<double> xc, yc, zc;
    std::vector<int> nEoC, EoC, CoC, VoC, CoE, VoE, EoV, CoV;
    std::vector<double> A, Av, kite, dc, dv, f, b;
};

struct RegionsHost {
    int M = 1, layers = 1;
    int order = 3;                                 // 2 = LTS2, 3 = LTS3
    // several disjoint fine regions (nreg > 1): the cells of region r's
    // bands F deep..C5 form block r-1 (band order inside), the far coarse
    // cells (C rest) the last block; mb*[k] = band offsets of block k as the
    // planner sees them (C rest empty for a region, only C rest for the
    // last block); Mr = each region's M.
    int nreg = 1;
    std::vector<int> Mr;
    std::vector<std::vector<int>> mcb, meb, mvb;   // [nreg + 1][NBANDS + 1]
    int ordering = 0;                              // 0 Hilbert inside a band, 1 mesh index order
    std::vector<int8_t> fine;                      // the fine-cell mask the labels came from
    std::vector<int8_t> rid;                       // region of each fine cell (several regions)
    std::vector<int8_t> cband, eband, vband;      // original order
    std::vector<int> perm_c, perm_e, perm_v;      // new -> original
    std::vector<int> inv_c, inv_e, inv_v;         // original -> new
    int cb[NBANDS + 1], eb[NBANDS + 1], vb[NBANDS + 1];   // band offsets (new order)
    // band-ordered connectivity (slot-major for cells)
    std::vector<uint8_t> cn;
    std::vector<int> se, sn, sv, ec0, ec1, vc, ve;
    std::vector<uint32_t> ep;
    // tiles of the fused kernel (see build_tiles)
    int tile_cells = 0;
    int ntiles = 0;
    int tb[NBANDS + 1];                         // first tile of each band
    std::vector<int4> tile_a;                   // {cell begin, own cells, halo begin, local cells}
    std::vector<int4> tile_b;                   // {edge begin, edge end, vert begin, local vertices}
    std::vector<int> tile_lsv_off;              // [ntiles] start of the tile's lsv block
    std::vector<int> halo;                      // halo cells of all tiles
    std::vector<int> tverts;                    // local vertex lists of all tiles
    std::vector<uint16_t> lsv;                  // per tile, slot-major: local vertex of (slot, local cell)
    std::vector<uint32_t> lec;                  // [nE] local cells of the owning tile: c0 | c1 << 16
    int max_local_cells = 0, max_local_verts = 0;
};

// Tiles of at most `tile_cells` consecutive cells of one band; a tile owns
// the edges whose lower band-order cell lies in it (a contiguous edge range).
int build_tiles(const HostMesh& m, RegionsHost& r, int tile_cells);

template <class T>
struct CoefTables {
    std::vector<T> snl, sR, sK, rA, b, rdc, db, vk, vd, f;
    std::vector<double> sK64, area, bd;
};

// Labels, bands and band-ordered connectivity.  ordering 0: Hilbert curve
// inside each band; 1: the mesh's own index order inside each band.
int compute_regions(const HostMesh& m, const int8_t* fine, int layers, int ordering, RegionsHost& r);
// Several fine regions: region_of_cell[i] = r in 1..nreg for the fine cells
// of region r, 0 elsewhere.  The regions' fine, interface, C1 and C2 cells
// must not touch (LTS_EINVAL otherwise).
int compute_regions_multi(const HostMesh& m, const int8_t* region_of_cell, int nreg, int layers, int ordering,
                          RegionsHost& r);
template <class T>
void coefficient_tables(const HostMesh& m, const RegionsHost& r, CoefTables<T>& o);
// The ring pass's packed slot rows (Tables::sidx, Tables::scf) from the
// slot-major index and coefficient arrays: {edge, neighbour, vertex, the
// bits of n l in FP32 (0 in FP64)} and, in FP32 only, {kite fraction, K
// coefficient}.  Every table set the ring kernel reads must carry them.
template <class T>
void pack_ring_slots(const std::vector<int>& se, const std::vector<int>& sn, const std::vector<int>& sv,
                     const std::vector<T>& snl, const std::vector<T>& sR, const std::vector<T>& sK,
                     std::vector<int4>& sidx, std::vector<float2>& scf);
// The edge and vertex passes' packed rows (Tables::erow, vri, vrd, vrk)
// from the plain edge arrays [nE] and the vertex arrays [3 nV] (entry k of
// vertex v at k nV + v) and f [nV]: {ec0, ec1, ep, the bits of rdc in FP32
// (0 in FP64)}, {ve0, ve1, ve2, vc0} and, in FP32 only, {vd0, vd1, vd2, f}
// and {vk0, vk1, vk2, the bits of vc1}.  Every table set the vertex and edge
// kernels read must carry them.
template <class T>
void pack_edge_vertex_rows(const std::vector<int>& ec0, const std::vector<int>& ec1,
                           const std::vector<uint32_t>& ep, const std::vector<T>& rdc, const std::vector<int>& vc,
                           const std::vector<int>& ve, const std::vector<T>& vd, const std::vector<T>& vk,
                           const std::vector<T>& f, std::vector<int4>& erow, std::vector<int4>& vri,
                           std::vector<float4>& vrd, std::vector<float4>& vrk);
double derived_weight(const HostMesh& m, int c, int j, int p);

}  // namespace lts
