// mesh_build.cpp -- seeded mesh generators (input generation only).
//
// Emits the MPAS-style arrays of Appendix B (cells = Voronoi generators,
// vertices = Delaunay triangles / Voronoi corners, edges = cell pairs) for
//   * a doubly periodic plane of regular hexagons, and
//   * a spherical centroidal Voronoi tessellation (SCVT) built by Lloyd
//     iteration on a density function from a seeded random start.
// The generators hold geometry and connectivity only: none of the method's
// arithmetic (no TRiSK weights, no operators, no time stepping) lives here.
//
// Geometry (Appendix B): x_v is the circumcentre of its Delaunay triangle,
// x_e the midpoint of the cell pair (where the cell-cell arc meets the
// vertex-vertex arc of a Voronoi diagram), d_e = the distance from x_c0 to
// x_c1 and l_e = the distance from x_v0 to x_v1 (great-circle arcs of
// radius R on the sphere, straight lines on the plane), kite (i, v) =
// signed area of (x_i, x_e1, x_v, x_e2),
// A_i = sum of the kites of cell i, A_v = sum of the kites at vertex v.
// Orientation: cellsOnEdge[2e] is the larger cell index (the Remark of
// Appendix B: i1 > i2 => n_{e,i1} = 1); verticesOnEdge[2e+1] is the left end.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <vector>

#include "../../include/lts.h"
#include "lts_error.h"

namespace {

constexpr double kOmega = 7.292e-5;
constexpr double kPi = 3.14159265358979323846;

struct V3 {
    double x, y, z;
};
inline V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 operator*(double s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
inline double norm(V3 a) { return std::sqrt(dot(a, a)); }
inline V3 unit(V3 a) { return (1.0 / norm(a)) * a; }

// ------------------------------------------------------------------ geometry
struct Geom {
    bool sphere;
    double R;        // sphere radius
    double Lx, Ly;   // plane periods

    V3 disp(V3 a, V3 b) const {  // plane: minimum-image b - a
        double dx = b.x - a.x, dy = b.y - a.y;
        dx -= Lx * std::floor(dx / Lx + 0.5);
        dy -= Ly * std::floor(dy / Ly + 0.5);
        return {dx, dy, 0.0};
    }
    V3 wrap(V3 a) const {
        return {a.x - Lx * std::floor(a.x / Lx), a.y - Ly * std::floor(a.y / Ly), 0.0};
    }
    // Unit-sphere positions on the sphere, metres on the plane.
    V3 circumcenter(V3 a, V3 b, V3 c) const {
        if (sphere) return unit(cross(b - a, c - a));
        V3 bb = disp(a, b), cc = disp(a, c);
        double d = 2.0 * (bb.x * cc.y - bb.y * cc.x);
        double b2 = dot(bb, bb), c2 = dot(cc, cc);
        V3 u{(cc.y * b2 - bb.y * c2) / d, (bb.x * c2 - cc.x * b2) / d, 0.0};
        return wrap(a + u);
    }
    double dist(V3 a, V3 b) const {
        if (sphere) return R * std::atan2(norm(cross(a, b)), dot(a, b));
        return norm(disp(a, b));
    }
    // Signed area, positive for counter-clockwise (seen from outside).
    double area(V3 a, V3 b, V3 c) const {
        if (sphere) {
            double num = dot(a, cross(b, c));
            double den = 1.0 + dot(a, b) + dot(b, c) + dot(c, a);
            return R * R * 2.0 * std::atan2(num, den);
        }
        V3 bb = disp(a, b), cc = disp(a, c);
        return 0.5 * (bb.x * cc.y - bb.y * cc.x);
    }
    V3 midpoint(V3 a, V3 b) const {
        if (sphere) return unit(a + b);
        return wrap(a + 0.5 * disp(a, b));
    }
};

template <class T>
T* dup_array(const std::vector<T>& v) {
    T* p = static_cast<T*>(std::malloc(std::max<size_t>(1, v.size()) * sizeof(T)));
    if (p && !v.empty()) std::memcpy(p, v.data(), v.size() * sizeof(T));
    return p;
}

// Builds the MPAS arrays from a triangulation of the generators.  `tri`
// lists counter-clockwise triangles (3 generator indices each) that tile the
// closed surface (sphere or torus).
int mesh_from_triangulation(const Geom& G, const std::vector<V3>& P, const std::vector<int>& tri,
                            double f0, lts_mesh_desc* out) {
    const int nC = static_cast<int>(P.size());
    const int nV = static_cast<int>(tri.size() / 3);
    // ---- edges: unique generator pairs, sorted by (min, max)
    struct Side {
        int lo, hi, t, k;
    };
    std::vector<Side> sides(3 * static_cast<size_t>(nV));
    for (int t = 0; t < nV; ++t)
        for (int k = 0; k < 3; ++k) {
            int a = tri[3 * t + k], b = tri[3 * t + (k + 1) % 3];
            sides[3 * t + k] = {std::min(a, b), std::max(a, b), t, k};
        }
    std::sort(sides.begin(), sides.end(), [](const Side& x, const Side& y) {
        return x.lo != y.lo ? x.lo < y.lo : (x.hi != y.hi ? x.hi < y.hi : x.t < y.t);
    });
    if (sides.size() % 2) return lts::set_error(LTS_EINVAL, "triangulation is not closed");
    const int nE = static_cast<int>(sides.size() / 2);
    std::vector<int> CoE(2 * static_cast<size_t>(nE)), VoE(2 * static_cast<size_t>(nE));
    std::vector<int> edge_of_side(3 * static_cast<size_t>(nV));
    for (int e = 0; e < nE; ++e) {
        const Side& s0 = sides[2 * e];
        const Side& s1 = sides[2 * e + 1];
        if (s0.lo != s1.lo || s0.hi != s1.hi || s0.lo == s0.hi)
            return lts::set_error(LTS_EINVAL, "triangulation side %d is not shared by two triangles", e);
        int c0 = s0.hi, c1 = s0.lo;  // n_e points out of the larger index
        CoE[2 * e] = c0;
        CoE[2 * e + 1] = c1;
        // The triangle that holds the directed side c0 -> c1 (counter-clockwise)
        // lies to the left of n_e, so its circumcentre is the left end.
        int ta = s0.t, ka = s0.k;
        int a0 = tri[3 * ta + ka];
        int tl = (a0 == c0) ? s0.t : s1.t;
        int tr = (tl == s0.t) ? s1.t : s0.t;
        VoE[2 * e] = tr;
        VoE[2 * e + 1] = tl;
        edge_of_side[3 * s0.t + s0.k] = e;
        edge_of_side[3 * s1.t + s1.k] = e;
    }
    // ---- per-vertex lists
    std::vector<int> EoV(3 * static_cast<size_t>(nV)), CoV(3 * static_cast<size_t>(nV));
    for (int t = 0; t < nV; ++t)
        for (int k = 0; k < 3; ++k) {
            CoV[3 * t + k] = tri[3 * t + k];
            EoV[3 * t + k] = edge_of_side[3 * t + k];
        }
    // ---- counter-clockwise rings of the cells
    // corner (t, k): at generator c = tri[t][k], neighbours a = tri[t][k+1], b = tri[t][k+2];
    // going counter-clockwise around c, a comes before b.
    std::vector<int> deg(nC, 0);
    for (int t = 0; t < nV; ++t)
        for (int k = 0; k < 3; ++k) deg[tri[3 * t + k]]++;
    std::vector<int> off(nC + 1, 0);
    for (int c = 0; c < nC; ++c) off[c + 1] = off[c] + deg[c];
    std::vector<int> corner(off[nC]);
    std::vector<int> fill(off.begin(), off.end() - 1);
    for (int t = 0; t < nV; ++t)
        for (int k = 0; k < 3; ++k) corner[fill[tri[3 * t + k]]++] = 3 * t + k;
    int maxE = 0;
    for (int c = 0; c < nC; ++c) maxE = std::max(maxE, deg[c]);
    if (maxE < 3) return lts::set_error(LTS_EINVAL, "degenerate triangulation");
    std::vector<int> nEoC(nC), EoC(static_cast<size_t>(nC) * maxE, -1),
        CoC(static_cast<size_t>(nC) * maxE, -1), VoC(static_cast<size_t>(nC) * maxE, -1);
    for (int c = 0; c < nC; ++c) {
        int n = deg[c];
        nEoC[c] = n;
        std::vector<char> used(n, 0);
        int cur = corner[off[c]];
        used[0] = 1;
        for (int j = 0; j < n; ++j) {
            int t = cur / 3, k = cur % 3;
            int a = tri[3 * t + (k + 1) % 3], b = tri[3 * t + (k + 2) % 3];
            EoC[static_cast<size_t>(c) * maxE + j] = edge_of_side[3 * t + k];  // side (c, a)
            CoC[static_cast<size_t>(c) * maxE + j] = a;
            VoC[static_cast<size_t>(c) * maxE + j] = t;
            if (j + 1 == n) break;
            int nxt = -1;
            for (int q = 0; q < n; ++q) {
                if (used[q]) continue;
                int cq = corner[off[c] + q];
                if (tri[3 * (cq / 3) + (cq % 3 + 1) % 3] == b) {
                    nxt = q;
                    break;
                }
            }
            if (nxt < 0) return lts::set_error(LTS_EINVAL, "cell %d has a broken ring", c);
            used[nxt] = 1;
            cur = corner[off[c] + nxt];
        }
    }
    // ---- geometry
    std::vector<V3> xv(nV), xe(nE);
    for (int t = 0; t < nV; ++t)
        xv[t] = G.circumcenter(P[tri[3 * t]], P[tri[3 * t + 1]], P[tri[3 * t + 2]]);
    std::vector<double> dc(nE), dv(nE);
    for (int e = 0; e < nE; ++e) {
        xe[e] = G.midpoint(P[CoE[2 * e]], P[CoE[2 * e + 1]]);
        dc[e] = G.dist(P[CoE[2 * e]], P[CoE[2 * e + 1]]);
        dv[e] = G.dist(xv[VoE[2 * e]], xv[VoE[2 * e + 1]]);
    }
    std::vector<double> kite(3 * static_cast<size_t>(nV), 0.0), Ac(nC, 0.0), Av(nV, 0.0);
    for (int c = 0; c < nC; ++c) {
        int n = nEoC[c];
        for (int j = 0; j < n; ++j) {
            int v = VoC[static_cast<size_t>(c) * maxE + j];
            int e1 = EoC[static_cast<size_t>(c) * maxE + j];
            int e2 = EoC[static_cast<size_t>(c) * maxE + (j + 1) % n];
            double k = G.area(P[c], xe[e1], xv[v]) + G.area(P[c], xv[v], xe[e2]);
            int slot = -1;
            for (int q = 0; q < 3; ++q)
                if (CoV[3 * v + q] == c) slot = q;
            kite[3 * v + slot] = k;
            Ac[c] += k;
        }
    }
    for (int v = 0; v < nV; ++v) Av[v] = kite[3 * v] + kite[3 * v + 1] + kite[3 * v + 2];
    std::vector<double> fv(nV);
    for (int v = 0; v < nV; ++v) fv[v] = G.sphere ? 2.0 * kOmega * xv[v].z : f0;

    // ---- output
    std::memset(out, 0, sizeof(*out));
    out->nCells = nC;
    out->nEdges = nE;
    out->nVertices = nV;
    out->maxEdges = maxE;
    out->on_sphere = G.sphere ? 1 : 0;
    out->radius = G.sphere ? G.R : 0.0;
    out->period_x = G.sphere ? 0.0 : G.Lx;
    out->period_y = G.sphere ? 0.0 : G.Ly;
    double s = G.sphere ? G.R : 1.0;
    auto split = [&](const std::vector<V3>& pts, double** x, double** y, double** z) {
        std::vector<double> a(pts.size()), b(pts.size()), c(pts.size());
        for (size_t i = 0; i < pts.size(); ++i) {
            a[i] = s * pts[i].x;
            b[i] = s * pts[i].y;
            c[i] = s * pts[i].z;
        }
        *x = dup_array(a);
        *y = dup_array(b);
        *z = dup_array(c);
    };
    split(P, &out->xCell, &out->yCell, &out->zCell);
    split(xe, &out->xEdge, &out->yEdge, &out->zEdge);
    split(xv, &out->xVertex, &out->yVertex, &out->zVertex);
    out->nEdgesOnCell = dup_array(nEoC);
    out->edgesOnCell = dup_array(EoC);
    out->cellsOnCell = dup_array(CoC);
    out->verticesOnCell = dup_array(VoC);
    out->cellsOnEdge = dup_array(CoE);
    out->verticesOnEdge = dup_array(VoE);
    out->edgesOnVertex = dup_array(EoV);
    out->cellsOnVertex = dup_array(CoV);
    out->areaCell = dup_array(Ac);
    out->areaTriangle = dup_array(Av);
    out->kiteAreasOnVertex = dup_array(kite);
    out->dcEdge = dup_array(dc);
    out->dvEdge = dup_array(dv);
    out->fVertex = dup_array(fv);
    if (!out->areaCell || !out->kiteAreasOnVertex || !out->cellsOnVertex) {
        lts_mesh_desc_free(out);
        return lts::set_error(LTS_ENOMEM, "out of host memory in the mesh builder");
    }
    return LTS_OK;
}

// --------------------------------------------------------- random numbers
// splitmix64 (Steele, Lea & Flood 2014) seeds xoshiro256** (Blackman & Vigna).
struct Rng {
    uint64_t s[4];
    explicit Rng(uint64_t seed) {
        uint64_t z = seed;
        for (auto& w : s) {
            z += 0x9e3779b97f4a7c15ULL;
            uint64_t x = z;
            x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ULL;
            x = (x ^ (x >> 27)) * 0x94d049bb133111ebULL;
            w = x ^ (x >> 31);
        }
    }
    static uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }
    uint64_t next() {
        uint64_t r = rotl(s[1] * 5, 7) * 9, t = s[1] << 17;
        s[2] ^= s[0];
        s[3] ^= s[1];
        s[1] ^= s[2];
        s[0] ^= s[3];
        s[2] ^= t;
        s[3] = rotl(s[3], 45);
        return r;
    }
    double uniform() { return (next() >> 11) * (1.0 / 9007199254740992.0); }
};

// ------------------------------------------------------------------ density
struct Density {
    lts_density d{};
    std::vector<V3> centres;
    explicit Density(const lts_density* rho) {
        if (rho) d = *rho;
        if (d.ncaps < 0) d.ncaps = 0;
        if (d.ncaps > 4) d.ncaps = 4;
        for (int k = 0; k < d.ncaps; ++k) {
            const lts_cap& c = d.cap[k];
            centres.push_back({std::cos(c.lat) * std::cos(c.lon), std::cos(c.lat) * std::sin(c.lon),
                               std::sin(c.lat)});
        }
    }
    // target spacing relative to the coarse spacing
    double spacing(V3 x) const {
        double s = 1.0;
        for (int k = 0; k < d.ncaps; ++k) {
            const lts_cap& c = d.cap[k];
            double ang = std::atan2(norm(cross(centres[k], x)), dot(centres[k], x));
            double r = c.ratio > 1.0 ? c.ratio : 1.0;
            double sk = 1.0 / r + (1.0 - 1.0 / r) * 0.5 * (1.0 + std::tanh((ang - c.radius) / c.width));
            s = std::min(s, sk);
        }
        return s;
    }
    double rho(V3 x) const {
        double s = spacing(x);
        return 1.0 / (s * s * s * s);
    }
    double min_spacing() const {
        double s = 1.0;
        for (int k = 0; k < d.ncaps; ++k)
            if (d.cap[k].ratio > 1.0) s = std::min(s, 1.0 / d.cap[k].ratio);
        return s;
    }
};

// ------------------------------------------------- spherical Delaunay (DT)
// Incremental insertion with Lawson flips (Lawson 1977; the sphere version
// of the planar algorithm).  Triangles are counter-clockwise seen from
// outside; tn[3t+k] is the neighbour across the side (v[k], v[k+1]).
struct SphDT {
    const std::vector<V3>* P = nullptr;
    std::vector<int> tv, tn;

    const V3& p(int i) const { return (*P)[i]; }
    int ntri() const { return static_cast<int>(tv.size() / 3); }

    // > 0 when d lies inside the circumcircle of the counter-clockwise (a,b,c)
    double incircle(int a, int b, int c, int d) const {
        V3 n = cross(p(b) - p(a), p(c) - p(a));
        V3 w = p(d) - p(a);
        double val = dot(n, w);
        double tol = 1e-12 * norm(n) * norm(w);
        return val > tol ? val : 0.0;
    }
    double left(int a, int b, V3 q) const { return dot(p(a), cross(p(b), q)); }

    void set(int t, int a, int b, int c, int na, int nb, int nc) {
        tv[3 * t] = a;
        tv[3 * t + 1] = b;
        tv[3 * t + 2] = c;
        tn[3 * t] = na;
        tn[3 * t + 1] = nb;
        tn[3 * t + 2] = nc;
    }
    void relink(int t, int from, int to) {
        if (t < 0) return;
        for (int k = 0; k < 3; ++k)
            if (tn[3 * t + k] == from) {
                tn[3 * t + k] = to;
                return;
            }
    }
    // Flip the side k of t if it is illegal; returns true if flipped.  After
    // a flip, t = (x, z, p') and u = (z, y, p') where (x, y) was the side.
    bool flip_if_illegal(int t, int k, std::vector<std::pair<int, int>>& stack) {
        int u = tn[3 * t + k];
        if (u < 0) return false;
        int x = tv[3 * t + k], y = tv[3 * t + (k + 1) % 3], q = tv[3 * t + (k + 2) % 3];
        int j = -1;
        for (int m = 0; m < 3; ++m)
            if (tv[3 * u + m] == y && tv[3 * u + (m + 1) % 3] == x) j = m;
        if (j < 0) return false;
        int z = tv[3 * u + (j + 2) % 3];
        if (incircle(x, y, q, z) <= 0.0) return false;
        int t_yq = tn[3 * t + (k + 1) % 3], t_qx = tn[3 * t + (k + 2) % 3];
        int u_xz = tn[3 * u + (j + 1) % 3], u_zy = tn[3 * u + (j + 2) % 3];
        set(t, x, z, q, u_xz, u, t_qx);
        set(u, z, y, q, u_zy, t_yq, t);
        relink(u_xz, u, t);
        relink(t_yq, t, u);
        stack.push_back({t, 0});
        stack.push_back({t, 2});
        stack.push_back({u, 0});
        stack.push_back({u, 1});
        return true;
    }
    void legalize(std::vector<std::pair<int, int>>& stack, int64_t max_flips) {
        int64_t flips = 0;
        while (!stack.empty() && flips < max_flips) {
            auto [t, k] = stack.back();
            stack.pop_back();
            if (flip_if_illegal(t, k, stack)) ++flips;
        }
    }
    int locate(V3 q, int t) const {
        int guard = 0;
        int rot = 0;
        while (guard++ < 100000000) {
            bool moved = false;
            for (int r = 0; r < 3; ++r) {
                int k = (r + rot) % 3;
                if (left(tv[3 * t + k], tv[3 * t + (k + 1) % 3], q) < 0.0) {
                    t = tn[3 * t + k];
                    moved = true;
                    break;
                }
            }
            rot = (rot + 1) % 3;
            if (!moved) return t;
        }
        return -1;
    }
    void insert(int pi, int t, std::vector<std::pair<int, int>>& stack) {
        int a = tv[3 * t], b = tv[3 * t + 1], c = tv[3 * t + 2];
        int nab = tn[3 * t], nbc = tn[3 * t + 1], nca = tn[3 * t + 2];
        int t1 = ntri(), t2 = ntri() + 1;
        tv.resize(tv.size() + 6);
        tn.resize(tn.size() + 6);
        set(t, a, b, pi, nab, t1, t2);
        set(t1, b, c, pi, nbc, t2, t);
        set(t2, c, a, pi, nca, t, t1);
        relink(nbc, t, t1);
        relink(nca, t, t2);
        stack.push_back({t, 0});
        stack.push_back({t1, 0});
        stack.push_back({t2, 0});
        legalize(stack, INT64_MAX);
    }

    // Build from scratch: initial tetrahedron + BRIO order of the rest.
    bool build(const std::vector<V3>& pts, uint64_t seed) {
        P = &pts;
        int n = static_cast<int>(pts.size());
        tv.clear();
        tn.clear();
        V3 dirs[4] = {{1, 1, 1}, {1, -1, -1}, {-1, 1, -1}, {-1, -1, 1}};
        int pick[4] = {-1, -1, -1, -1};
        double best[4] = {-2, -2, -2, -2};
        for (int i = 0; i < n; ++i)
            for (int k = 0; k < 4; ++k) {
                double d = dot(pts[i], unit(dirs[k]));
                if (d > best[k]) {
                    best[k] = d;
                    pick[k] = i;
                }
            }
        for (int k = 0; k < 4; ++k)
            for (int m = k + 1; m < 4; ++m)
                if (pick[k] == pick[m]) return false;
        // four faces, each counter-clockwise seen from outside
        int f[4][3] = {{pick[0], pick[1], pick[2]}, {pick[0], pick[3], pick[1]},
                       {pick[1], pick[3], pick[2]}, {pick[0], pick[2], pick[3]}};
        int opp[4] = {pick[3], pick[2], pick[0], pick[1]};
        tv.resize(12);
        tn.assign(12, -1);
        for (int k = 0; k < 4; ++k) {
            V3 a = pts[f[k][0]], b = pts[f[k][1]], c = pts[f[k][2]];
            double o = dot(cross(b - a, c - a), pts[opp[k]] - a);
            if (o > 0) std::swap(f[k][1], f[k][2]);
            a = pts[f[k][0]];
            b = pts[f[k][1]];
            c = pts[f[k][2]];
            if (dot(cross(b - a, c - a), V3{0, 0, 0} - a) >= 0) return false;  // origin inside
            for (int m = 0; m < 3; ++m) tv[3 * k + m] = f[k][m];
        }
        for (int t = 0; t < 4; ++t)
            for (int k = 0; k < 3; ++k) {
                int a = tv[3 * t + k], b = tv[3 * t + (k + 1) % 3];
                for (int u = 0; u < 4; ++u)
                    for (int m = 0; m < 3; ++m)
                        if (tv[3 * u + m] == b && tv[3 * u + (m + 1) % 3] == a) tn[3 * t + k] = u;
            }
        // BRIO: random rounds of doubling size, Morton order inside a round
        std::vector<int> order;
        order.reserve(n);
        for (int i = 0; i < n; ++i)
            if (i != pick[0] && i != pick[1] && i != pick[2] && i != pick[3]) order.push_back(i);
        Rng rng(seed ^ 0x5eedULL);
        for (size_t i = order.size(); i > 1; --i) std::swap(order[i - 1], order[rng.next() % i]);
        auto morton = [&](int i) {
            auto spread = [](uint64_t v) {
                v &= 0x1fffff;
                v = (v | v << 32) & 0x1f00000000ffffULL;
                v = (v | v << 16) & 0x1f0000ff0000ffULL;
                v = (v | v << 8) & 0x100f00f00f00f00fULL;
                v = (v | v << 4) & 0x10c30c30c30c30c3ULL;
                v = (v | v << 2) & 0x1249249249249249ULL;
                return v;
            };
            auto q = [](double c) { return static_cast<uint64_t>((c + 1.0) * 0.5 * 2097151.0); };
            return spread(q(pts[i].x)) | (spread(q(pts[i].y)) << 1) | (spread(q(pts[i].z)) << 2);
        };
        size_t start = 0, len = std::min<size_t>(order.size(), 64);
        while (start < order.size()) {
            size_t end = std::min(order.size(), start + len);
            std::sort(order.begin() + start, order.begin() + end,
                      [&](int a, int b) { return morton(a) < morton(b); });
            start = end;
            len *= 2;
        }
        tv.reserve(6 * static_cast<size_t>(n));
        tn.reserve(6 * static_cast<size_t>(n));
        std::vector<std::pair<int, int>> stack;
        int last = 0;
        for (int i : order) {
            int t = locate(pts[i], last);
            if (t < 0) return false;
            insert(i, t, stack);
            last = ntri() - 1;
        }
        return ntri() == 2 * n - 4;
    }
    // After the points moved: true if every triangle is still counter-clockwise.
    bool valid() const {
        for (int t = 0; t < ntri(); ++t)
            if (dot(p(tv[3 * t]), cross(p(tv[3 * t + 1]), p(tv[3 * t + 2]))) <= 0.0) return false;
        return true;
    }
    void flip_all() {
        std::vector<std::pair<int, int>> stack;
        for (int t = 0; t < ntri(); ++t)
            for (int k = 0; k < 3; ++k)
                if (tn[3 * t + k] > t) stack.push_back({t, k});
        legalize(stack, 50LL * ntri());
    }
};

// Density-weighted centroids of the Voronoi regions (Lloyd step): each
// region is split into the triangles (x_i, x_v(j), x_v(j+1)); every
// triangle contributes rho(m) * area * m with m its normalised centroid.
void lloyd_step(const SphDT& dt, const Density& den, std::vector<V3>& P) {
    const int n = static_cast<int>(P.size());
    const int T = dt.ntri();
    std::vector<V3> cc(T);
#pragma omp parallel for schedule(static)
    for (int t = 0; t < T; ++t) {
        V3 a = P[dt.tv[3 * t]], b = P[dt.tv[3 * t + 1]], c = P[dt.tv[3 * t + 2]];
        cc[t] = unit(cross(b - a, c - a));
    }
    std::vector<int> one(n, -1);
    for (int t = 0; t < T; ++t)
        for (int k = 0; k < 3; ++k) one[dt.tv[3 * t + k]] = 3 * t + k;
    Geom G{true, 1.0, 0.0, 0.0};
    std::vector<V3> next(n);
#pragma omp parallel for schedule(dynamic, 1024)
    for (int i = 0; i < n; ++i) {
        int t0 = one[i] / 3, k0 = one[i] % 3;
        int t = t0, k = k0;
        V3 acc{0, 0, 0};
        int guard = 0;
        do {
            // next triangle counter-clockwise around i: across side (v[k+2], v[k])
            int u = dt.tn[3 * t + (k + 2) % 3];
            int m = 0;
            while (dt.tv[3 * u + m] != i) ++m;
            double A = G.area(P[i], cc[t], cc[u]);
            V3 mid = unit(P[i] + cc[t] + cc[u]);
            acc = acc + (den.rho(mid) * A) * mid;
            t = u;
            k = m;
        } while (t != t0 && ++guard < 64);
        next[i] = unit(acc);
    }
    P.swap(next);
}

}  // namespace

extern "C" {

void lts_mesh_desc_free(lts_mesh_desc* d) {
    if (!d) return;
    double** dp[] = {&d->xCell, &d->yCell, &d->zCell, &d->xEdge, &d->yEdge, &d->zEdge,
                     &d->xVertex, &d->yVertex, &d->zVertex, &d->areaCell, &d->areaTriangle,
                     &d->kiteAreasOnVertex, &d->dcEdge, &d->dvEdge, &d->fVertex, &d->bottom,
                     &d->weightsOnEdge};
    for (auto p : dp) {
        std::free(*p);
        *p = nullptr;
    }
    int32_t** ip[] = {&d->nEdgesOnCell, &d->edgesOnCell, &d->cellsOnCell, &d->verticesOnCell,
                      &d->cellsOnEdge, &d->verticesOnEdge, &d->edgesOnVertex, &d->cellsOnVertex,
                      &d->nEdgesOnEdge, &d->edgesOnEdge};
    for (auto p : ip) {
        std::free(*p);
        *p = nullptr;
    }
    std::memset(d, 0, sizeof(*d));
}

int lts_build_hex_periodic(int32_t nx, int32_t ny, double dc, double f0, lts_mesh_desc* out) {
    if (!out) return lts::set_error(LTS_EINVAL, "out is NULL");
    if (nx < 4 || ny < 4 || (ny % 2) != 0 || !(dc > 0.0))
        return lts::set_error(LTS_EINVAL, "hex mesh needs nx,ny >= 4, ny even, dc > 0 (got %d, %d, %g)",
                              nx, ny, dc);
    const double h = std::sqrt(3.0) / 2.0 * dc;
    Geom G{false, 0.0, nx * dc, ny * h};
    const int n = nx * ny;
    std::vector<V3> P(n);
    auto id = [&](int i, int j) {
        i = ((i % nx) + nx) % nx;
        j = ((j % ny) + ny) % ny;
        return j * nx + i;
    };
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) P[id(i, j)] = {(i + 0.5 * (j & 1)) * dc, j * h, 0.0};
    std::vector<int> tri;
    tri.reserve(6 * static_cast<size_t>(n));
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int c = id(i, j), E = id(i + 1, j);
            int NE = (j & 1) ? id(i + 1, j + 1) : id(i, j + 1);
            int NW = (j & 1) ? id(i, j + 1) : id(i - 1, j + 1);
            tri.insert(tri.end(), {c, E, NE, c, NE, NW});
        }
    return mesh_from_triangulation(G, P, tri, f0, out);
}

int lts_build_scvt(int64_t n, uint64_t seed, const lts_density* rho, int32_t lloyd_iters,
                   double radius, lts_mesh_desc* out) {
    if (!out) return lts::set_error(LTS_EINVAL, "out is NULL");
    if (n < 12 || n > (int64_t)1 << 28 || !(radius > 0.0) || lloyd_iters < 0)
        return lts::set_error(LTS_EINVAL, "scvt needs n >= 12, radius > 0, lloyd_iters >= 0");
    Density den(rho);
    Rng rng(seed);
    // seeded random start with point density rho^(1/2) (SCVT spacing ~ rho^(-1/4))
    const double smin = den.min_spacing();
    std::vector<V3> P;
    P.reserve(n);
    while (static_cast<int64_t>(P.size()) < n) {
        double z = 2.0 * rng.uniform() - 1.0;
        double phi = 2.0 * kPi * rng.uniform();
        double r = std::sqrt(std::max(0.0, 1.0 - z * z));
        V3 x{r * std::cos(phi), r * std::sin(phi), z};
        double s = den.spacing(x);
        double accept = (smin / s) * (smin / s);
        if (rng.uniform() < accept) P.push_back(x);
    }
    SphDT dt;
    if (!dt.build(P, seed)) return lts::set_error(LTS_EINVAL, "spherical Delaunay build failed");
    for (int it = 0; it < lloyd_iters; ++it) {
        lloyd_step(dt, den, P);
        dt.P = &P;
        if (dt.valid()) {
            dt.flip_all();
        } else if (!dt.build(P, seed + it + 1)) {
            return lts::set_error(LTS_EINVAL, "spherical Delaunay rebuild failed at iteration %d", it);
        }
    }
    if (!dt.valid() && !dt.build(P, seed + 7)) return lts::set_error(LTS_EINVAL, "final rebuild failed");
    Geom G{true, radius, 0.0, 0.0};
    return mesh_from_triangulation(G, P, dt.tv, 0.0, out);
}

}  // extern "C"
