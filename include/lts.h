/*
 * lts.h -- C ABI of liblts.so: local time stepping (LTS3) for the TRiSK
 * C-grid shallow-water equations on a Voronoi mesh, on one GB300 GPU.
 *
 * Method: Capodaglio & Petersen, "Local time stepping for the shallow water
 * equations in MPAS" (arXiv:2106.07154), Section 2 (Algorithms 2.1 and 2.2,
 * index sets of Eqs. (3)-(5)) and Appendix B (TRiSK operators).
 *
 * Conventions shared by every entry point
 *  - Return value: LTS_OK (0) or a negative LTS_E* code; a message for the
 *    last failure of the calling thread is in lts_last_error().  No C++
 *    exception crosses this boundary.
 *  - The caller owns every array it passes; the library copies what it keeps.
 *    Arrays are host memory unless the name says otherwise.
 *  - Indices are 0-based int32.  Lengths in metres, times in seconds.
 *  - Orientation: the normal n_e of edge e points out of cellsOnEdge[2e+0]
 *    (n_{e,i} = +1 for that cell, Appendix B) and verticesOnEdge[2e+1] is
 *    the vertex in direction k x n_e (t_{e,v} = +1).  The mesh builders set
 *    cellsOnEdge[2e+0] to the larger of the two cell indices, the rule of the
 *    Remark in Appendix B.  The library never re-derives the orientation:
 *    normal velocities u_e keep the caller's sign convention on input and
 *    on output.
 *  - Handles are opaque and owned by the library; destroy them with the
 *    matching lts_*_destroy.  A state holds its mesh and regions alive
 *    (reference counted), so destroy order does not matter.
 */
#ifndef LTS_H
#define LTS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LTS_OK          0
#define LTS_EINVAL     -1   /* bad argument, size or mesh                      */
#define LTS_ENOMEM     -2   /* host or device allocation failed                */
#define LTS_ECUDA      -3   /* a CUDA runtime call failed (message says which) */
#define LTS_ENONFINITE -4   /* a thickness became <= 0 or non-finite           */
#define LTS_ETIMEOUT   -5   /* a bounded device wait gave up                   */
#define LTS_ENODEV     -6   /* no usable CUDA device                           */

/* ------------------------------------------------------------------------
 * Mesh description (MPAS-style arrays, host memory).
 *   Appendix B: cells (Voronoi generators) carry h, b, K; edges carry the
 *   normal velocity u_e; vertices (dual triangles) carry q_v.
 *   l_e = dvEdge (primal edge length), d_e = dcEdge (cell-to-cell distance),
 *   A_i = areaCell, A_v = areaTriangle, A_{i,v} = kiteAreasOnVertex.
 * Layout: edgesOnCell/cellsOnCell/verticesOnCell are [nCells*maxEdges],
 *   listed counter-clockwise; verticesOnCell[i*maxEdges+j] lies between
 *   edgesOnCell[..+j] and edgesOnCell[..+j+1] (mod nEdgesOnCell[i]);
 *   cellsOnCell[..+j] is the neighbour across edgesOnCell[..+j].
 *   cellsOnEdge/verticesOnEdge are [nEdges*2]; edgesOnVertex/cellsOnVertex/
 *   kiteAreasOnVertex are [nVertices*3] (kite k belongs to cellsOnVertex k).
 * Optional arrays may be NULL: positions, bottom (flat), edgesOnEdge,
 *   nEdgesOnEdge, weightsOnEdge ([nEdges*2*maxEdges]; if present they are
 *   checked against the weights the library derives from the kite areas).
 * Builders fill every required array with malloc'ed memory; free it with
 *   lts_mesh_desc_free.  A caller-filled desc is never freed by the library.
 * ------------------------------------------------------------------------ */
typedef struct lts_mesh_desc {
    int32_t nCells, nEdges, nVertices, maxEdges;
    int32_t on_sphere;               /* 1: sphere of `radius`; 0: doubly periodic plane */
    double radius;                   /* sphere radius [m]                                */
    double period_x, period_y;       /* plane periods [m]                                */
    double *xCell, *yCell, *zCell;   /* [nCells]     Cartesian positions (z = 0 on plane) */
    double *xEdge, *yEdge, *zEdge;   /* [nEdges]     x_e                                  */
    double *xVertex, *yVertex, *zVertex; /* [nVertices]                                   */
    int32_t *nEdgesOnCell;           /* [nCells]                                          */
    int32_t *edgesOnCell, *cellsOnCell, *verticesOnCell; /* [nCells*maxEdges]             */
    int32_t *cellsOnEdge, *verticesOnEdge;               /* [nEdges*2]                    */
    int32_t *edgesOnVertex, *cellsOnVertex;              /* [nVertices*3]                 */
    double *areaCell;                /* [nCells]    A_i                                   */
    double *areaTriangle;            /* [nVertices] A_v                                   */
    double *kiteAreasOnVertex;       /* [nVertices*3] A_{i,v}                             */
    double *dcEdge, *dvEdge;         /* [nEdges]    d_e, l_e                              */
    double *fVertex;                 /* [nVertices] Coriolis parameter f_v                */
    double *bottom;                  /* [nCells]    bottom topography b_i (NULL = 0)      */
    int32_t *nEdgesOnEdge, *edgesOnEdge;  /* optional MPAS tables                         */
    double *weightsOnEdge;                /* optional, w_{e,e'} of Appendix B Eq. (weights) */
} lts_mesh_desc;

/* One refined cap of a spherical density function.  The target spacing is
 * s(x) = min over caps of  1/ratio + (1 - 1/ratio) (1 + tanh((d - radius)/width))/2
 * (relative to the coarse spacing, d = great-circle angle from the cap
 * centre) and the SCVT density is rho = s^-4, so `ratio` is the
 * coarse-to-fine resolution ratio.  Angles in radians. */
typedef struct lts_cap {
    double lon, lat, radius, width, ratio;
} lts_cap;

typedef struct lts_density {
    int32_t ncaps;                   /* 0 = uniform density                               */
    lts_cap cap[4];
} lts_density;

/* Doubly periodic plane of regular hexagons (Appendix B geometry with
 * x_e at the cell-pair midpoint).  nx*ny cells, cell spacing dc [m],
 * Coriolis parameter f0 (f-plane).  ny must be even, nx,ny >= 4.
 * Cells are numbered row by row.  Errors: LTS_EINVAL, LTS_ENOMEM. */
int lts_build_hex_periodic(int32_t nx, int32_t ny, double dc, double f0,
                           lts_mesh_desc* out);

/* Spherical centroidal Voronoi tessellation (SCVT) with n generators on a
 * sphere of `radius` (the variable-resolution SCVT meshes of the test cases
 * in Section 3, which the paper takes from MPAS; seeded stand-ins here), made by `lloyd_iters` Lloyd iterations from a seeded
 * random start drawn with point density rho^(1/2) (rho from `rho`, NULL =
 * uniform).  Voronoi vertices are circumcentres of the spherical Delaunay
 * triangles; kite areas are signed spherical areas of (x_i, x_e1, x_v, x_e2);
 * f_v = 2 Omega sin(lat_v) with Omega = 7.292e-5 s^-1.  Host only, uses
 * OpenMP threads.  Errors: LTS_EINVAL (n < 12, radius <= 0), LTS_ENOMEM. */
int lts_build_scvt(int64_t n, uint64_t seed, const lts_density* rho,
                   int32_t lloyd_iters, double radius, lts_mesh_desc* out);

/* Frees the arrays a builder allocated and zeroes the struct (memory
 * management; the paper has no counterpart). */
void lts_mesh_desc_free(lts_mesh_desc* d);

/* ------------------------------------------------------------------------
 * Device objects.
 * ------------------------------------------------------------------------ */
typedef struct lts_mesh_s* lts_mesh;
typedef struct lts_regions_s* lts_regions;
typedef struct lts_state_s* lts_state;

/* Validates and copies the mesh of Appendix B (its arrays, the orientation
 * rule of its Remark, and the weights of its Eq. (weights)); the FP64
 * master copies stay on the host until regions are set.  Checks index ranges, orientation consistency, positive
 * areas and lengths, kite sums (sum over a cell = A_i, over a vertex = A_v,
 * relative 1e-9) and, if given, weightsOnEdge against the kite-derived
 * weights (absolute 1e-9).  Errors: LTS_EINVAL, LTS_ENOMEM. */
int lts_mesh_create(const lts_mesh_desc* d, lts_mesh* out);
void lts_mesh_destroy(lts_mesh m);

/* Region labelling of Eqs. (3)-(5) from a fine-cell mask ([nCells], nonzero
 * = F^c), then band ordering: cells sorted by band
 *   0 F deep | 1 F3 | 2 F2 | 3 F1 | 4 I1 | 5 I2 | 6 C1 | 7 C2 | 8 C3 | 9 C4 |
 *   10 C5 | 11 C rest
 * (F1,F2 = the two fine layers of Eq. (4); F3 = the next fine layer; C1..C5 =
 * the five coarse layers next to I2) and by a Hilbert curve inside each
 * band; an edge takes the smaller band of its two cells (the fine-to-coarse
 * assignment of Eq. (5)), a vertex the smallest band of its three cells.
 * Every restricted phase then reads and writes contiguous index ranges.
 * Host only: the first lts_state_create of each precision uploads the
 * band-ordered device tables (FP64 master geometry, FP32/FP64 coefficient
 * copies derived in FP64 and rounded once).
 *   order:            3 (LTS3) or 2 (LTS2, the second-order branches of
 *                     Algorithm 2.2); other values -> LTS_EINVAL.
 *   M:                fine substeps per coarse step, >= 1.
 *   interface_layers: cells per interface layer (>= 1): I1 = cells at
 *                     edge-distance 1..L from F, I2 = distance L+1..2L.
 * Errors: LTS_EINVAL, LTS_ENOMEM. */
int lts_regions_set(lts_mesh m, const int8_t* fine_mask, int32_t order, int32_t M,
                    int32_t interface_layers, lts_regions* out);
void lts_regions_destroy(lts_regions r);

/* Several disjoint fine regions, each with its own M, sharing the coarse
 * step (the more-than-two-regions case of the Remark in Section 2.3, for
 * regions that are not nested): Steps 1, 2 and 4 of Algorithm 2.2 run on
 * the union of the sets; Step 3 and Step 5 run per region r with M[r-1] on
 * its own fine and interface sets.  region_of_cell[i] = r in 1..nregions
 * for the fine cells of region r, 0 elsewhere.  Each region's cells of the
 * bands F..C5 form one contiguous block (band order and Hilbert order
 * inside), the far coarse cells a last block; the plans of the blocks merge
 * launch by launch into segment-table launches.  A region's fine,
 * interface and first two coarse layers must not touch another region's
 * (LTS_EINVAL).  LTS3 only (order 3); three-launch path, one layer, no
 * profiling, no fused tiles.  nregions = 1 is lts_regions_set. */
int lts_regions_set_multi(lts_mesh m, const int8_t* region_of_cell, int32_t nregions,
                          const int32_t* M, int32_t order, int32_t interface_layers,
                          lts_regions* out);

/* Region labels of Eqs. (3)-(5) in the caller's original order (host
 * arrays):
 *   cell_label [nCells]: 0 F \ Fbar, 1 F2, 2 F1, 3 I1, 4 I2, 5 C
 *   edge_label [nEdges]: 0 F^e, 1 Fbar^e, 3 I1^e, 4 I2^e, 5 C^e
 * Either pointer may be NULL. */
int lts_regions_labels(lts_regions r, int8_t* cell_label, int8_t* edge_label);

/* Re-tiles the regions for the fused kernel (kernel_path = 1): tiles of at
 * most tile_cells consecutive band-order cells (32..4096; default 256).  A
 * GPU layout choice; the paper has no counterpart.
 * Only while no state uses the regions.  Errors: LTS_EINVAL. */
int lts_regions_tiling(lts_regions r, int32_t tile_cells);

/* Order of the cells inside each band (the bands themselves are fixed; a
 * memory layout choice that replaces the paper's METIS partitioning of
 * Section 3.1, so the paper has no counterpart):
 *   LTS_ORDER_HILBERT (default): along a Hilbert curve through the cell
 *     centres, so neighbours sit close in memory;
 *   LTS_ORDER_INDEX: the mesh's own index order (the naive layout, for
 *     comparison).
 * Edges and vertices follow their cells.  Only while no state uses the
 * regions.  Every element's arithmetic is the same in either order, so
 * results are identical; only the memory access pattern changes.
 * Errors: LTS_EINVAL, LTS_ENOMEM. */
#define LTS_ORDER_HILBERT 0
#define LTS_ORDER_INDEX   1
int lts_regions_ordering(lts_regions r, int32_t ordering);

/* Number of cells, edges and vertices per band (arrays of LTS_NBANDS): the
 * sizes of the index sets of Eqs. (3)-(5) split by band. */
#define LTS_NBANDS 12
int lts_regions_counts(lts_regions r, int64_t* cells, int64_t* edges, int64_t* vertices);

/* Band-order permutations: perm_cell[new] = original index (any may be
 * NULL).  A memory layout; the paper has no counterpart. */
int lts_regions_permutation(lts_regions r, int32_t* perm_cell, int32_t* perm_edge,
                            int32_t* perm_vertex);

#define LTS_FP32 0
#define LTS_FP64 1
#define LTS_MODE_LTS    0   /* Algorithm 2.2 of the regions' order (LTS2 or LTS3),
                               coarse step dt, M from the regions                    */
#define LTS_MODE_LTS3   0   /* the same value (the regions' order decides)           */
#define LTS_MODE_SSPRK3 1   /* Algorithm 2.1 (SSPRK3) on the whole mesh, step dt    */
#define LTS_MODE_SSPRK2 2   /* Algorithm 2.1 (SSPRK2) on the whole mesh, step dt    */

#define LTS_COARSE_FAR    0   /* the default */
#define LTS_COARSE_STEP4  1
#define LTS_COARSE_SERIAL 2

typedef struct lts_params {
    double g;               /* gravity [m s^-2]                                        */
    double dt;              /* coarse step (LTS3) or step (SSPRK3) [s]                 */
    int32_t precision;      /* LTS_FP32 or LTS_FP64                                    */
    int32_t mode;           /* LTS_MODE_LTS, LTS_MODE_SSPRK3 or LTS_MODE_SSPRK2        */
    int32_t compensated;    /* FP32: carry a compensation word with every state value
                               (stage sums and flux divergence compensated); ignored
                               for FP64                                                */
    int32_t use_graph;      /* 1: capture one coarse step as a CUDA graph (default)    */
    int32_t block_size;     /* threads per block, 0 = library default                 */
    int32_t profile;        /* 1: CUDA events around every direct launch (no graph);
                               2: event-record nodes around every kernel node of the
                               graph (per-kernel times of the last lts_step call)      */
    int32_t pdl;            /* 1: programmatic dependent launch between consecutive
                               kernels (each launch overlaps its predecessor's tail)   */
    int32_t kernel_path;    /* 0: three launches per right-hand side (vertex PV, cell
                               ring, edge; default); 1: one fused tile kernel per
                               right-hand side (shared-memory staging per tile)        */
    void* stream;           /* cudaStream_t to enqueue on; NULL = a library stream     */
    int32_t no_l2_hints;    /* 1: table loads without L2 eviction priorities (default:
                               keep the fine region, stream the coarse one)            */
    int32_t layers;         /* independent shallow-water layers advanced on the same
                               mesh (0 or 1 = one).  The paper's speed-up runs repeat
                               every computation for 100 layers to model an ocean
                               workload; here the layers share every mesh-table load.
                               h0/u0, lts_read and lts_write then take [layers][nCells]
                               and [layers][nEdges] (layer-major, original order inside
                               a layer); diagnostics sum over the layers.  Three-launch
                               path only, no ensembles.                                */
    int32_t ring_occupancy; /* FP32, three-launch path: 0 (default) or 6 / 8 = the ring
                               pass built for that many resident 256-thread blocks per
                               SM (fewer registers, some spills), leaving block slots
                               for the next launch's table prefetch                   */
    int32_t coarse_schedule;/* order of the coarse phases (results are identical):
                               LTS_COARSE_FAR (default): Steps 1, 2 and 4 on the far
                               coarse bands (C5+ for Step 1, C3+ for Steps 2 and 4)
                               run as a concurrent graph branch beside Step 3 (LTS2
                               and the fused path: Step 4 / the last coarse stage
                               only); LTS_COARSE_STEP4: only Step 4 on C3+ forms that
                               branch; LTS_COARSE_SERIAL: step order on one stream     */
    int32_t elems_per_thread;/* vertex and edge launches of single-layer states on the
                               three-launch path: 1 or 2 elements per thread (2: half
                               the blocks, both elements' loads in flight together);
                               0 = library default.  Results are identical.            */
} lts_params;

/* Allocates the device state (band order) and uploads (h0, u0), the
 * thickness and normal velocity of Eq. (1), given in the caller's original
 * order ([nCells], [nEdges], FP64 host arrays), for the integrator p->mode
 * selects (Algorithm 2.2, or Algorithm 2.1 on the whole mesh).  Captures
 * the CUDA graphs of one coarse step when use_graph = 1 (so create the state
 * outside any stream capture).  Errors: LTS_EINVAL (dt <= 0, g <= 0, bad
 * precision/mode), LTS_ENOMEM, LTS_ECUDA. */
int lts_state_create(lts_mesh m, lts_regions r, const double* h0, const double* u0,
                     const lts_params* p, lts_state* out);
void lts_state_destroy(lts_state s);

/* Enqueues n_coarse coarse steps (Algorithm 2.2, Steps 1-5, with the
 * regions' M fine substeps in Step 3; its LTS2 branches for order-2 regions)
 * or steps (Algorithm 2.1: SSPRK3 or SSPRK2) on the state's stream.  Every
 * stage evaluates the right-hand side of Eq. (1) with the operators of
 * Appendix B on the sets the step names.  Asynchronous: returns after
 * enqueueing.  n_coarse >= 0. */
int lts_step(lts_state s, int32_t n_coarse);

/* Autotuner: times candidate launch configurations of one coarse step on
 * scratch states built from (m, r, h0, u0) and *base, and returns the
 * fastest as *best (base's g, dt, precision, mode, compensation and stream
 * kept; use_graph = 1).  Candidates: block_size 128 or 256, kernel_path 0
 * or 1, pdl on or off, L2 hints on or off, the coarse schedule (LTS3:
 * LTS_COARSE_FAR, _STEP4 or _SERIAL; LTS2: _FAR or _SERIAL).  Each is timed over `steps` coarse
 * steps after 3 warm-up steps; the three fastest are timed twice more and
 * the best of three wins.  With the winner, FP32 states also try the ring
 * occupancy variants 6 and 8, and single-region single-layer states the
 * other elems_per_thread (best of two timings each).  With
 * flags & LTS_TUNE_ORDERING and no state using r, the other cell ordering
 * (lts_regions_ordering) is tried with the winner and r keeps the faster.
 * No configuration changes a result bit; the tuner only chooses speed.  The
 * paper has no counterpart (it runs with MPI defaults).  Needs a CUDA
 * device; synchronises.  rep may be NULL.
 * Errors: LTS_EINVAL (bad arguments, nothing buildable), LTS_ENOMEM,
 * LTS_ECUDA. */
#define LTS_TUNE_ORDERING 1
typedef struct lts_tune_entry {
    int32_t block_size, kernel_path, pdl, l2_hints, coarse_schedule, ordering, ring_occupancy,
            elems_per_thread;
    double ms;              /* ms per coarse step (best of its timings; inf = not buildable) */
} lts_tune_entry;
typedef struct lts_tune_report {
    int32_t candidates;     /* configurations timed                              */
    int32_t ordering;       /* cell ordering r has afterwards (LTS_ORDER_*)      */
    double best_ms;         /* ms per coarse step of *best                       */
    double default_ms;      /* ms per coarse step of the library defaults        */
    lts_tune_entry entry[32];   /* the first min(candidates, 32) timings          */
} lts_tune_report;
int lts_autotune(lts_mesh m, lts_regions r, const double* h0, const double* u0,
                 const lts_params* base, int32_t steps, int32_t flags, lts_params* best,
                 lts_tune_report* rep);

typedef struct lts_diag {
    double mass;            /* sum_i A_i h_i (FP64 reduction of the FP64 or FP32+compensation state) */
    double energy;          /* sum_i A_i h_i (K_i + g (h_i/2 + b_i))                               */
    double time;            /* simulated time [s]                                                  */
    int64_t steps;          /* coarse steps taken                                                  */
} lts_diag;

/* Synchronises the state's stream and copies the state (h, u) of Eq. (1)
 * to the caller in the original order and orientation (h [nCells], u [nEdges], FP64; either may
 * be NULL), plus diagnostics (d may be NULL).  Returns LTS_ENONFINITE if any
 * stage produced a thickness <= 0 or a non-finite value since the last read
 * or lts_sync.  Equivalent to lts_read_async followed by lts_sync. */
int lts_read(lts_state s, double* h, double* u, lts_diag* d);

/* Replaces the state (original order, FP64 host arrays), e.g. to resume from
 * a saved lts_read (checkpoint and restart; the paper has no counterpart); `time`/`steps` set the clock.  Enqueued: the copies run
 * on a host-to-device stream of the state as soon as the previous write's
 * staging is free (they may overlap coarse steps enqueued earlier), and the
 * state is replaced in stream order.  From pageable memory the call returns
 * once the data is staged; from pinned memory it returns at once, and the
 * caller keeps h and u unchanged until the next lts_sync or lts_read. */
int lts_write(lts_state s, const double* h, const double* u, double time, int64_t steps);

/* Streaming host I/O (the paper has no counterpart; an interface for moving
 * a state in and out every step, e.g. many independent states through one
 * solver).  lts_read_async enqueues the copy of the state as it stands after
 * everything enqueued so far into h, u (original order, FP64; either may be
 * NULL) and, with d, its diagnostics, and returns at once.  The state is
 * gathered on the state's stream and copied on a device-to-host stream, so
 * the copy overlaps coarse steps enqueued after it.  h, u and *d are valid
 * after the next lts_sync (or lts_read), and must stay allocated until then
 * (the library writes them); use pinned memory for the overlap.
 * At most 16 reads with diagnostics between two syncs (LTS_EINVAL beyond).
 * lts_sync waits for all the state's work and copies, and returns
 * LTS_ENONFINITE as lts_read does.  Errors: LTS_EINVAL, LTS_ECUDA. */
int lts_read_async(lts_state s, double* h, double* u, lts_diag* d);
int lts_sync(lts_state s);

/* Launch statistics of one coarse step (measurement; the paper has no
 * counterpart): number of kernel launches, and per
 * launch kind k (0 = vertex PV, 1 = cell ring pass with the thickness
 * update, 2 = edge pass with the velocity update, 3 = fused tile kernel
 * doing all three for a tile) the algorithmic bytes
 * summed over the step (each array element a launch touches counted once).
 * With profile = 1, ms[k] is the summed event time of those launches in the
 * last lts_step call (0 otherwise).  Arrays of LTS_NKINDS. */
#define LTS_NKINDS 4
int lts_step_stats(lts_state s, int32_t* launches_per_step, double* bytes, double* ms,
                   int32_t* launches_per_kind);

/* Mass and energy of the current state (the FP64 reduction lts_read
 * performs, with the same blocking, so the sums agree to the last bit), for
 * callers that cannot allocate device memory when they need them: hosts
 * whose device memory comes from a fixed pool that must not grow, or time
 * loops that forbid allocation because cudaMalloc may synchronise the
 * device.  The paper has no counterpart; this is an interface convenience.
 *   d_out: device memory owned by the caller, 2 doubles: {mass, energy}.
 * Allocates nothing: the per-block partial sums live in one fixed device
 * array of 4096 x 2 doubles (64 KiB) inside liblts.so, which every GPU that
 * loads the library keeps until the process exits; states of more than
 * 4096 * 256 = 1,048,576 cells x layers are rejected with LTS_EINVAL before
 * anything is enqueued.  The first call on a device looks the array's
 * address up (cudaGetSymbolAddress), so make that first call before any
 * stream capture.  Enqueued on the state's stream, no synchronisation.  All
 * calls share the array, and every call overwrites the partial sums it
 * reads, so calls that overlap on the GPU (different streams, unordered)
 * race and must not be issued.
 * Errors: LTS_EINVAL (null argument, state too large, state on another
 * device), LTS_ECUDA. */
int lts_diagnostics_noalloc(lts_state s, double* d_out);

/* ------------------------------------------------------------------------
 * Ensembles: several independent states (each its own mesh, regions, M and
 * dt) advanced together, one launch per phase of the coarse step for all
 * members (the phases of Algorithm 2.2, or of 2.1 for SSPRK3 members).
 * The paper runs one mesh per job; batching independent meshes is an
 * interface of this library.  The members' tables and states are copied
 * into one packed index space; each launch carries the segments (band
 * ranges) of every member in a device table (each block finds its segment),
 * and a member with a smaller M has no segments in the later substeps.
 * Every member's cells see the same arithmetic as its stand-alone
 * lts_step, so results equal the members' own steps bit for bit.
 * ------------------------------------------------------------------------ */
typedef struct lts_ensemble_s* lts_ensemble;

typedef struct lts_ensemble_params {
    int32_t use_graph;      /* 1: capture one ensemble coarse step as a CUDA graph     */
    int32_t pdl;            /* 1: programmatic dependent launch between launches       */
    int32_t persistent;     /* 1: grid = resident blocks, each walking the pieces;
                               0: one block per 256-element piece of a segment
                               (default; the faster of the two on GB300)               */
    void* stream;           /* cudaStream_t to enqueue on; NULL = a library stream     */
} lts_ensemble_params;

/* Builds an ensemble (the paper has no counterpart) of n >= 1 distinct states that live on the current
 * device and share precision, compensation, mode, g, block size and
 * kernel_path 0.  Copies each member's current state in (the members'
 * streams are synchronised first).  p may be NULL (graph, PDL, one block
 * per piece).
 * The members must outlive the ensemble and must not be stepped, written
 * or destroyed while it exists; lts_ensemble_read brings a member's own
 * state up to date.  Needs at most 2^31 - 1 cells x maxEdges in total.
 * Errors: LTS_EINVAL, LTS_ENOMEM, LTS_ECUDA, LTS_ENODEV. */
int lts_ensemble_create(const lts_state* members, int32_t n, const lts_ensemble_params* p,
                        lts_ensemble* out);
void lts_ensemble_destroy(lts_ensemble e);

/* Enqueues n_coarse coarse steps of every member (each with its own dt and
 * M; Algorithm 2.2 or 2.1 per member, as lts_step) on the ensemble's
 * stream; asynchronous.  n_coarse >= 0. */
int lts_ensemble_step(lts_ensemble e, int32_t n_coarse);

/* Ensemble I/O (the paper has no counterpart).
 * Copies member i's packed state into the member (its clock advanced by
 * the ensemble's steps), then behaves as lts_read on that member.  Returns
 * LTS_ENONFINITE if any member produced a thickness <= 0 or a non-finite
 * value since the last ensemble read (the flag is shared by all members). */
int lts_ensemble_read(lts_ensemble e, int32_t i, double* h, double* u, lts_diag* d);

/* Asynchronous member read (as lts_read_async on the member; the paper has
 * no counterpart): enqueues the
 * unpacking of member i and the copy of its state to h, u (and *d), which
 * are valid after lts_ensemble_sync and must stay allocated until then;
 * pinned memory overlaps the copies with
 * later work.  lts_ensemble_sync waits for the ensemble and every member,
 * and returns LTS_ENONFINITE as lts_ensemble_read does.  Keep host buffers
 * that a later lts_ensemble_write reads unchanged until the sync. */
int lts_ensemble_read_async(lts_ensemble e, int32_t i, double* h, double* u, lts_diag* d);
int lts_ensemble_sync(lts_ensemble e);

/* Replaces member i's state (original order, FP64 host arrays, as
 * lts_write; the paper has no counterpart) inside the ensemble, e.g. to restart one member; `time` and
 * `steps` set that member's clock.  Enqueued: the ensemble's stream waits
 * for the member's copy (an event, no host synchronisation); from pinned
 * memory the caller keeps h and u unchanged until the next
 * lts_ensemble_read. */
int lts_ensemble_write(lts_ensemble e, int32_t i, const double* h, const double* u, double time,
                       int64_t steps);

/* Launches and segment records per ensemble coarse step (measurement; the
 * paper has no counterpart), algorithmic bytes
 * per launch kind (array of LTS_NKINDS, summed over members), and the total
 * number of cells.  Any pointer may be NULL. */
int lts_ensemble_stats(lts_ensemble e, int32_t* launches_per_step, double* bytes, int64_t* cells,
                       int32_t* segments_per_step);

/* Message of the calling thread's last failure (error reporting; the paper
 * has no counterpart). */
const char* lts_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
