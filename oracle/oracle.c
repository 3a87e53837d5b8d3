/*
 * oracle.c -- plain, slow FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).
 *
 * Implements, in the paper's order and notation:
 *   - the TRiSK operators of Appendix B (thickness flux, divergence, gradient,
 *     kinetic energy, vertex potential vorticity, the weights w_{e,e'} of
 *     Eq. (weights) and the potential-vorticity flux F^perp_e [q]_{v->e}),
 *   - the semi-discrete system of Eq. (1),
 *   - Algorithm 2.1 (SSPRK3), classical RK4 (the reference-solution
 *     generator of Section 3.2) and Algorithm 2.2 (LTS3),
 *   - the index sets of Eqs. (3)-(5).
 * Every right-hand side is evaluated on the whole mesh in the original index
 * order; results are written only to the index sets the algorithm names.
 * There is no blocking, fusion or reordering.
 *
 * Readings of the paper where it is silent, garbled or inconsistent:
 *  R1 (Eq. 5, garbled): Fbar^e = {edges of Fbar^c cells} \ F^e.  Step 3
 *     advances the fine edges F^e u Fbar^e (all edges of F^c cells that are
 *     not interface edges); Step 3's initialisation covers the same set.
 *  R2 (Steps 3.3.3 and 4 print 2/3 h^{1st}): SSPRK3's third stage,
 *     1/3 x^{old} + 2/3 x^{2nd} + 2/3 dt RHS(x^{2nd}), with dt/M in Step 3.
 *  R3 (Steps 3.2.3, 3.3.3 drop the ",k" superscripts): read old -> old,k,
 *     1st -> 1st,k, 2nd -> 2nd,k on the fine sets.
 *  R4 (values outside F u I1 during Step 3): the stage vectors keep the
 *     coarse stage values (old / 1st / 2nd) there for every k; only I1 is
 *     predicted.
 *  R5 (Step 5): evaluated as the Shu-Osher replay of the three interface
 *     stages, x1 = x_old + (dt/M) H1, x2 = 3/4 x_old + 1/4 x1 + 1/4 (dt/M) H2,
 *     x_new = 1/3 x_old + 2/3 x2 + 2/3 (dt/M) H3, which is algebraically
 *     identical to Step 5 (theta = 1/6, 1/6, 2/3) and makes M = 1 reproduce
 *     SSPRK3 bit for bit; the printed form is available as step5_form = 1.
 *  R6 (Eq. 3 read literally lets F cells be "interface" too): I1 excludes
 *     F, I2 excludes F u I1, F2 excludes F1.
 *  R7 (q_v undefined): zeta_v = (1/A_v) sum_{e in EV(v)} t_{e,v} d_e u_e,
 *     h_v = (1/A_v) sum_{i in CV(v)} A_{i,v} h_i, q_v = (zeta_v + f_v) / h_v.
 *  R8 (energy not defined): E = sum_i A_i h_i (K_i + g (h_i/2 + b_i)).
 */
#include "oracle.h"

#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

struct or_mesh {
    int nC, nE, nV, maxE;
    int *nEoC, *EoC;        /* EC(i) */
    int *CoE, *VoE;         /* CE(e), VE(e) */
    int *EoV, *CoV;         /* EV(v), CV(v) */
    double *A, *Av, *kite, *dc, *dv, *f, *b;
    /* EE(e) and w_{e,e'} (Eq. weights), built once from the arrays above */
    int *nEE, *EE;
    double *W;
};

static void* xmalloc(size_t n) { return malloc(n ? n : 1); }

static int* dup_i(const int* p, size_t n) {
    int* q = (int*)xmalloc(n * sizeof(int));
    memcpy(q, p, n * sizeof(int));
    return q;
}
static double* dup_d(const double* p, size_t n) {
    double* q = (double*)xmalloc(n * sizeof(double));
    if (p) memcpy(q, p, n * sizeof(double));
    else memset(q, 0, n * sizeof(double));
    return q;
}

/* n_{e,i} of Appendix B: +1 if n_e is an outward normal of cell i. */
static double n_sign(const or_mesh* m, int e, int i) {
    return (m->CoE[2 * e] == i) ? 1.0 : -1.0;
}
/* t_{e,v} of Appendix B: +1 if v is at the left end of e (direction k x n_e). */
static double t_sign(const or_mesh* m, int e, int v) {
    return (m->VoE[2 * e + 1] == v) ? 1.0 : -1.0;
}
/* Kite area A_{i,v}. */
static double kite_area(const or_mesh* m, int i, int v) {
    for (int k = 0; k < 3; ++k)
        if (m->CoV[3 * v + k] == i) return m->kite[3 * v + k];
    return 0.0;
}
/* The vertex shared by two edges of the same cell that follow each other. */
static int shared_vertex(const or_mesh* m, int ea, int eb) {
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            if (m->VoE[2 * ea + a] == m->VoE[2 * eb + b]) return m->VoE[2 * ea + a];
    return -1;
}

/* Eq. (weights): for e' in EE(e) with common cell i*, walk from e' to e
 * along the edges of i* (the order of edgesOnCell; Appendix B allows either
 * sense), collect the vertices met, v* the last one, and set
 * w_{e,e'} = n_{e',i*} t_{e,v*} (sum_{v} A_{i*,v}/A_{i*} - 1/2). */
static double trisk_weight(const or_mesh* m, int e, int ep, int cell) {
    int n = m->nEoC[cell];
    const int* ec = m->EoC + (size_t)cell * m->maxE;
    int jp = -1, je = -1;
    for (int j = 0; j < n; ++j) {
        if (ec[j] == ep) jp = j;
        if (ec[j] == e) je = j;
    }
    if (jp < 0 || je < 0) return 0.0;
    double sum = 0.0;
    int vstar = -1;
    for (int j = jp; j != je; j = (j + 1) % n) {
        int v = shared_vertex(m, ec[j], ec[(j + 1) % n]);
        sum += kite_area(m, cell, v) / m->A[cell];
        vstar = v;
    }
    return n_sign(m, ep, cell) * t_sign(m, e, vstar) * (sum - 0.5);
}

static void build_weights(or_mesh* m) {
    int w = 2 * m->maxE;
    m->nEE = (int*)xmalloc((size_t)m->nE * sizeof(int));
    m->EE = (int*)xmalloc((size_t)m->nE * w * sizeof(int));
    m->W = (double*)xmalloc((size_t)m->nE * w * sizeof(double));
    for (int e = 0; e < m->nE; ++e) {
        int cnt = 0;
        for (int s = 0; s < 2; ++s) {
            int cell = m->CoE[2 * e + s];
            for (int j = 0; j < m->nEoC[cell]; ++j) {
                int ep = m->EoC[(size_t)cell * m->maxE + j];
                if (ep == e) continue;
                m->EE[(size_t)e * w + cnt] = ep;
                m->W[(size_t)e * w + cnt] = trisk_weight(m, e, ep, cell);
                ++cnt;
            }
        }
        m->nEE[e] = cnt;
    }
}

or_mesh* or_mesh_new(int nCells, int nEdges, int nVertices, int maxEdges,
                     const int* nEdgesOnCell, const int* edgesOnCell,
                     const int* cellsOnEdge, const int* verticesOnEdge,
                     const int* edgesOnVertex, const int* cellsOnVertex,
                     const double* areaCell, const double* areaTriangle,
                     const double* kiteAreasOnVertex, const double* dcEdge,
                     const double* dvEdge, const double* fVertex,
                     const double* bottom) {
    if (nCells <= 0 || nEdges <= 0 || nVertices <= 0 || maxEdges <= 0) return NULL;
    for (int i = 0; i < nCells; ++i) {
        if (nEdgesOnCell[i] < 3 || nEdgesOnCell[i] > maxEdges) return NULL;
        for (int j = 0; j < nEdgesOnCell[i]; ++j) {
            int e = edgesOnCell[(size_t)i * maxEdges + j];
            if (e < 0 || e >= nEdges) return NULL;
        }
    }
    for (int e = 0; e < 2 * nEdges; ++e) {
        if (cellsOnEdge[e] < 0 || cellsOnEdge[e] >= nCells) return NULL;
        if (verticesOnEdge[e] < 0 || verticesOnEdge[e] >= nVertices) return NULL;
    }
    for (int v = 0; v < 3 * nVertices; ++v) {
        if (edgesOnVertex[v] < 0 || edgesOnVertex[v] >= nEdges) return NULL;
        if (cellsOnVertex[v] < 0 || cellsOnVertex[v] >= nCells) return NULL;
    }
    or_mesh* m = (or_mesh*)calloc(1, sizeof(or_mesh));
    m->nC = nCells; m->nE = nEdges; m->nV = nVertices; m->maxE = maxEdges;
    m->nEoC = dup_i(nEdgesOnCell, nCells);
    m->EoC = dup_i(edgesOnCell, (size_t)nCells * maxEdges);
    m->CoE = dup_i(cellsOnEdge, 2 * (size_t)nEdges);
    m->VoE = dup_i(verticesOnEdge, 2 * (size_t)nEdges);
    m->EoV = dup_i(edgesOnVertex, 3 * (size_t)nVertices);
    m->CoV = dup_i(cellsOnVertex, 3 * (size_t)nVertices);
    m->A = dup_d(areaCell, nCells);
    m->Av = dup_d(areaTriangle, nVertices);
    m->kite = dup_d(kiteAreasOnVertex, 3 * (size_t)nVertices);
    m->dc = dup_d(dcEdge, nEdges);
    m->dv = dup_d(dvEdge, nEdges);
    m->f = dup_d(fVertex, nVertices);
    m->b = dup_d(bottom, nCells);
    build_weights(m);
    return m;
}

void or_mesh_free(or_mesh* m) {
    if (!m) return;
    free(m->nEoC); free(m->EoC); free(m->CoE); free(m->VoE); free(m->EoV); free(m->CoV);
    free(m->A); free(m->Av); free(m->kite); free(m->dc); free(m->dv); free(m->f); free(m->b);
    free(m->nEE); free(m->EE); free(m->W);
    free(m);
}

void or_weights(const or_mesh* m, int* neoe, int* eoe, double* woe) {
    int w = 2 * m->maxE;
    memcpy(neoe, m->nEE, (size_t)m->nE * sizeof(int));
    memcpy(eoe, m->EE, (size_t)m->nE * w * sizeof(int));
    memcpy(woe, m->W, (size_t)m->nE * w * sizeof(double));
}

/* ---------------------------------------------------------------- operators */

/* F_e = [h]_{i->e} u_e with [h]_{i->e} = 1/2 sum_{i in CE(e)} h_i. */
void or_thickness_flux(const or_mesh* m, const double* h, const double* u, double* F) {
#pragma omp parallel for schedule(static)
    for (int e = 0; e < m->nE; ++e) {
        double he = 0.5 * (h[m->CoE[2 * e]] + h[m->CoE[2 * e + 1]]);
        F[e] = he * u[e];
    }
}

/* [div F]_i = (1/A_i) sum_{e in EC(i)} n_{e,i} l_e F_e. */
void or_divergence(const or_mesh* m, const double* F, double* div) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < m->nC; ++i) {
        double s = 0.0;
        for (int j = 0; j < m->nEoC[i]; ++j) {
            int e = m->EoC[(size_t)i * m->maxE + j];
            s += n_sign(m, e, i) * m->dv[e] * F[e];
        }
        div[i] = s / m->A[i];
    }
}

/* [grad phi]_e = (1/d_e) sum_{i in CE(e)} -n_{e,i} phi_i. */
void or_gradient(const or_mesh* m, const double* phi, double* grad) {
#pragma omp parallel for schedule(static)
    for (int e = 0; e < m->nE; ++e) {
        double s = 0.0;
        for (int k = 0; k < 2; ++k) {
            int i = m->CoE[2 * e + k];
            s += -n_sign(m, e, i) * phi[i];
        }
        grad[e] = s / m->dc[e];
    }
}

/* K_i = 1/(4 A_i) sum_{e in EC(i)} l_e d_e u_e^2. */
void or_kinetic(const or_mesh* m, const double* u, double* K) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < m->nC; ++i) {
        double s = 0.0;
        for (int j = 0; j < m->nEoC[i]; ++j) {
            int e = m->EoC[(size_t)i * m->maxE + j];
            s += m->dv[e] * m->dc[e] * u[e] * u[e];
        }
        K[i] = s / (4.0 * m->A[i]);
    }
}

/* zeta_v = (1/A_v) sum_{e in EV(v)} t_{e,v} d_e u_e (circulation of the dual
 * cell divided by its area; reading R7). */
void or_vorticity(const or_mesh* m, const double* u, double* zeta) {
#pragma omp parallel for schedule(static)
    for (int v = 0; v < m->nV; ++v) {
        double s = 0.0;
        for (int k = 0; k < 3; ++k) {
            int e = m->EoV[3 * v + k];
            s += t_sign(m, e, v) * m->dc[e] * u[e];
        }
        zeta[v] = s / m->Av[v];
    }
}

/* q_v = (zeta_v + f_v) / h_v, h_v = (1/A_v) sum_{i in CV(v)} A_{i,v} h_i (R7). */
void or_pv_vertex(const or_mesh* m, const double* h, const double* u, double* q) {
    double* zeta = (double*)xmalloc((size_t)m->nV * sizeof(double));
    or_vorticity(m, u, zeta);
#pragma omp parallel for schedule(static)
    for (int v = 0; v < m->nV; ++v) {
        double hv = 0.0;
        for (int k = 0; k < 3; ++k) hv += m->kite[3 * v + k] * h[m->CoV[3 * v + k]];
        hv = hv / m->Av[v];
        q[v] = (zeta[v] + m->f[v]) / hv;
    }
    free(zeta);
}

/* F_e^perp = sum_{e' in EE(e)} w_{e,e'} (l_{e'}/d_e) F_{e'}. */
void or_tangential(const or_mesh* m, const double* F, double* Fperp) {
    int w = 2 * m->maxE;
#pragma omp parallel for schedule(static)
    for (int e = 0; e < m->nE; ++e) {
        double s = 0.0;
        for (int j = 0; j < m->nEE[e]; ++j) {
            int ep = m->EE[(size_t)e * w + j];
            s += m->W[(size_t)e * w + j] * (m->dv[ep] / m->dc[e]) * F[ep];
        }
        Fperp[e] = s;
    }
}

/* F_e^perp [q]_{v->e} = sum_{e' in EE(e)} w_{e,e'} (l_{e'}/d_e) F_{e'} (qt_e + qt_{e'})/2,
 * with qt_e = 1/2 sum_{v in VE(e)} q_v supplied as qe. */
void or_pv_flux(const or_mesh* m, const double* F, const double* qe, double* pv) {
    int w = 2 * m->maxE;
#pragma omp parallel for schedule(static)
    for (int e = 0; e < m->nE; ++e) {
        double s = 0.0;
        for (int j = 0; j < m->nEE[e]; ++j) {
            int ep = m->EE[(size_t)e * w + j];
            s += m->W[(size_t)e * w + j] * (m->dv[ep] / m->dc[e]) * F[ep] *
                 (qe[e] + qe[ep]) / 2.0;
        }
        pv[e] = s;
    }
}

/* Eq. (1): H_i = -[div F]_i,  U_e = -F_e^perp [q]_{v->e} - [g grad(h+b) + grad K]_e. */
void or_rhs_swe(const or_mesh* m, double g, const double* h, const double* u,
                double* H, double* U) {
    int nC = m->nC, nE = m->nE, nV = m->nV;
    double* F = (double*)xmalloc((size_t)nE * sizeof(double));
    double* q = (double*)xmalloc((size_t)nV * sizeof(double));
    double* qe = (double*)xmalloc((size_t)nE * sizeof(double));
    double* K = (double*)xmalloc((size_t)nC * sizeof(double));
    double* hb = (double*)xmalloc((size_t)nC * sizeof(double));
    double* div = (double*)xmalloc((size_t)nC * sizeof(double));
    double* ghb = (double*)xmalloc((size_t)nE * sizeof(double));
    double* gK = (double*)xmalloc((size_t)nE * sizeof(double));
    double* pv = (double*)xmalloc((size_t)nE * sizeof(double));

    or_thickness_flux(m, h, u, F);
    or_pv_vertex(m, h, u, q);
    for (int e = 0; e < nE; ++e) qe[e] = 0.5 * (q[m->VoE[2 * e]] + q[m->VoE[2 * e + 1]]);
    or_kinetic(m, u, K);
    for (int i = 0; i < nC; ++i) hb[i] = h[i] + m->b[i];
    or_divergence(m, F, div);
    or_gradient(m, hb, ghb);
    or_gradient(m, K, gK);
    or_pv_flux(m, F, qe, pv);
    for (int i = 0; i < nC; ++i) H[i] = -div[i];
    for (int e = 0; e < nE; ++e) U[e] = -pv[e] - (g * ghb[e] + gK[e]);

    free(F); free(q); free(qe); free(K); free(hb); free(div); free(ghb); free(gK); free(pv);
}

void or_rhs(const or_mesh* m, const or_system* sys, const double* h, const double* u,
            double* H, double* U) {
    if (sys->kind == OR_SYS_LINEAR) {
        for (int i = 0; i < m->nC; ++i) H[i] = sys->lam_c[i] * h[i];
        for (int e = 0; e < m->nE; ++e) U[e] = sys->lam_e[e] * u[e];
    } else {
        or_rhs_swe(m, sys->g, h, u, H, U);
    }
}

/* ---------------------------------------------------------------- regions */

/* Eqs. (3)-(5) with readings R1 and R6. */
/* One sweep of Eq. (3)'s "shares at least one edge with": every cell that
 * shares an edge with a marked cell becomes marked (synchronously). */
static void or_grow(const or_mesh* m, char* mark, char* tmp) {
    memcpy(tmp, mark, (size_t)m->nC);
    for (int e = 0; e < m->nE; ++e) {
        int a = m->CoE[2 * e], b = m->CoE[2 * e + 1];
        if (mark[a]) tmp[b] = 1;
        if (mark[b]) tmp[a] = 1;
    }
    memcpy(mark, tmp, (size_t)m->nC);
}

int or_regions(const or_mesh* m, const signed char* fine, signed char* cl, signed char* el) {
    return or_regions_layers(m, fine, 1, cl, el);
}

int or_regions_layers(const or_mesh* m, const signed char* fine, int L, signed char* cl,
                      signed char* el) {
    if (L < 1) return -1;
    int nC = m->nC, nE = m->nE;
    char* inF = (char*)calloc(nC, 1);
    char* inI1 = (char*)calloc(nC, 1);
    char* inI2 = (char*)calloc(nC, 1);
    char* inF1 = (char*)calloc(nC, 1);
    char* inF2 = (char*)calloc(nC, 1);
    char* reach = (char*)calloc(nC, 1);
    char* tmp = (char*)calloc(nC, 1);
    for (int i = 0; i < nC; ++i) inF[i] = fine[i] != 0;
    /* I1: not fine, reached from F by 1..L edge crossings (L = 1: shares an
     * edge with a fine cell, Eq. 3) */
    memcpy(reach, inF, (size_t)nC);
    for (int k = 0; k < L; ++k) or_grow(m, reach, tmp);
    for (int i = 0; i < nC; ++i) inI1[i] = reach[i] && !inF[i];
    /* I2: neither fine nor I1, reached from I1 by 1..L further crossings */
    for (int k = 0; k < L; ++k) or_grow(m, reach, tmp);
    for (int i = 0; i < nC; ++i) inI2[i] = reach[i] && !inF[i] && !inI1[i];
    free(reach);
    free(tmp);
    /* F1: fine, shares an edge with an I1 cell */
    for (int e = 0; e < nE; ++e) {
        int a = m->CoE[2 * e], b = m->CoE[2 * e + 1];
        if (inF[a] && inI1[b]) inF1[a] = 1;
        if (inF[b] && inI1[a]) inF1[b] = 1;
    }
    /* F2: fine, not F1, shares an edge with an F1 cell */
    for (int e = 0; e < nE; ++e) {
        int a = m->CoE[2 * e], b = m->CoE[2 * e + 1];
        if (inF[a] && !inF1[a] && inF1[b]) inF2[a] = 1;
        if (inF[b] && !inF1[b] && inF1[a]) inF2[b] = 1;
    }
    for (int i = 0; i < nC; ++i) {
        if (inF[i]) cl[i] = inF1[i] ? 2 : (inF2[i] ? 1 : 0);
        else if (inI1[i]) cl[i] = 3;
        else if (inI2[i]) cl[i] = 4;
        else cl[i] = 5;
    }
    /* Edge sets, assigned from the fine to the coarse side. */
    char* eF = (char*)calloc(nE, 1);
    char* eFb = (char*)calloc(nE, 1);
    char* eI1 = (char*)calloc(nE, 1);
    char* eI2 = (char*)calloc(nE, 1);
    for (int i = 0; i < nC; ++i) {
        for (int j = 0; j < m->nEoC[i]; ++j) {
            int e = m->EoC[(size_t)i * m->maxE + j];
            if (cl[i] == 0) eF[e] = 1;                  /* edges of F \ Fbar cells */
        }
    }
    for (int i = 0; i < nC; ++i) {
        for (int j = 0; j < m->nEoC[i]; ++j) {
            int e = m->EoC[(size_t)i * m->maxE + j];
            if ((cl[i] == 1 || cl[i] == 2) && !eF[e]) eFb[e] = 1;   /* Fbar^e */
        }
    }
    for (int i = 0; i < nC; ++i) {
        for (int j = 0; j < m->nEoC[i]; ++j) {
            int e = m->EoC[(size_t)i * m->maxE + j];
            if (cl[i] == 3 && !eFb[e]) eI1[e] = 1;      /* I1^e = edges(I1) \ Fbar^e */
        }
    }
    for (int i = 0; i < nC; ++i) {
        for (int j = 0; j < m->nEoC[i]; ++j) {
            int e = m->EoC[(size_t)i * m->maxE + j];
            if (cl[i] == 4 && !eI1[e]) eI2[e] = 1;      /* I2^e = edges(I2) \ I1^e */
        }
    }
    for (int e = 0; e < nE; ++e) {
        if (eF[e]) el[e] = 0;
        else if (eFb[e]) el[e] = 1;
        else if (eI1[e]) el[e] = 3;
        else if (eI2[e]) el[e] = 4;
        else el[e] = 5;                                 /* C^e = edges(C) \ I2^e */
    }
    free(inF); free(inI1); free(inI2); free(inF1); free(inF2);
    free(eF); free(eFb); free(eI1); free(eI2);
    return 0;
}

/* ------------------------------------------------------ SSP stage helpers */

/* Algorithm 2.1, the three SSPRK3 stages (omega_old = 3/4, omega_1st =
 * omega_rhs = 1/4).  Every integrator below goes through these three. */
static double ssp_stage1(double x_old, double rhs, double dt) {
    return x_old + dt * rhs;
}
static double ssp_stage2(double x_old, double x_1st, double rhs, double dt) {
    return 0.75 * x_old + 0.25 * x_1st + 0.25 * dt * rhs;
}
static double ssp_stage3(double x_old, double x_2nd, double rhs, double dt) {
    return (1.0 / 3.0) * x_old + (2.0 / 3.0) * x_2nd + (2.0 / 3.0) * dt * rhs;
}

void or_ssprk3(const or_mesh* m, const or_system* sys, double dt, int nsteps,
               double* h, double* u) {
    int nC = m->nC, nE = m->nE;
    double *h1 = xmalloc(nC * sizeof(double)), *u1 = xmalloc(nE * sizeof(double));
    double *h2 = xmalloc(nC * sizeof(double)), *u2 = xmalloc(nE * sizeof(double));
    double *H = xmalloc(nC * sizeof(double)), *U = xmalloc(nE * sizeof(double));
    for (int n = 0; n < nsteps; ++n) {
        or_rhs(m, sys, h, u, H, U);
        for (int i = 0; i < nC; ++i) h1[i] = ssp_stage1(h[i], H[i], dt);
        for (int e = 0; e < nE; ++e) u1[e] = ssp_stage1(u[e], U[e], dt);
        or_rhs(m, sys, h1, u1, H, U);
        for (int i = 0; i < nC; ++i) h2[i] = ssp_stage2(h[i], h1[i], H[i], dt);
        for (int e = 0; e < nE; ++e) u2[e] = ssp_stage2(u[e], u1[e], U[e], dt);
        or_rhs(m, sys, h2, u2, H, U);
        for (int i = 0; i < nC; ++i) h[i] = ssp_stage3(h[i], h2[i], H[i], dt);
        for (int e = 0; e < nE; ++e) u[e] = ssp_stage3(u[e], u2[e], U[e], dt);
    }
    free(h1); free(u1); free(h2); free(u2); free(H); free(U);
}

void or_rk4(const or_mesh* m, const or_system* sys, double dt, int nsteps,
            double* h, double* u) {
    int nC = m->nC, nE = m->nE;
    double *ht = xmalloc(nC * sizeof(double)), *ut = xmalloc(nE * sizeof(double));
    double *k1h = xmalloc(nC * sizeof(double)), *k1u = xmalloc(nE * sizeof(double));
    double *k2h = xmalloc(nC * sizeof(double)), *k2u = xmalloc(nE * sizeof(double));
    double *k3h = xmalloc(nC * sizeof(double)), *k3u = xmalloc(nE * sizeof(double));
    double *k4h = xmalloc(nC * sizeof(double)), *k4u = xmalloc(nE * sizeof(double));
    for (int n = 0; n < nsteps; ++n) {
        or_rhs(m, sys, h, u, k1h, k1u);
        for (int i = 0; i < nC; ++i) ht[i] = h[i] + 0.5 * dt * k1h[i];
        for (int e = 0; e < nE; ++e) ut[e] = u[e] + 0.5 * dt * k1u[e];
        or_rhs(m, sys, ht, ut, k2h, k2u);
        for (int i = 0; i < nC; ++i) ht[i] = h[i] + 0.5 * dt * k2h[i];
        for (int e = 0; e < nE; ++e) ut[e] = u[e] + 0.5 * dt * k2u[e];
        or_rhs(m, sys, ht, ut, k3h, k3u);
        for (int i = 0; i < nC; ++i) ht[i] = h[i] + dt * k3h[i];
        for (int e = 0; e < nE; ++e) ut[e] = u[e] + dt * k3u[e];
        or_rhs(m, sys, ht, ut, k4h, k4u);
        for (int i = 0; i < nC; ++i)
            h[i] += dt / 6.0 * (k1h[i] + 2.0 * k2h[i] + 2.0 * k3h[i] + k4h[i]);
        for (int e = 0; e < nE; ++e)
            u[e] += dt / 6.0 * (k1u[e] + 2.0 * k2u[e] + 2.0 * k3u[e] + k4u[e]);
    }
    free(ht); free(ut); free(k1h); free(k1u); free(k2h); free(k2u);
    free(k3h); free(k3u); free(k4h); free(k4u);
}

/* Algorithm 2.1 with SSPRK2: omega_old = omega_1st = omega_rhs = 1/2. */
static double ssp2_stage2(double x_old, double x_1st, double rhs, double dt) {
    return 0.5 * x_old + 0.5 * x_1st + 0.5 * dt * rhs;
}

void or_ssprk2(const or_mesh* m, const or_system* sys, double dt, int nsteps,
               double* h, double* u) {
    int nC = m->nC, nE = m->nE;
    double *h1 = xmalloc(nC * sizeof(double)), *u1 = xmalloc(nE * sizeof(double));
    double *H = xmalloc(nC * sizeof(double)), *U = xmalloc(nE * sizeof(double));
    for (int n = 0; n < nsteps; ++n) {
        or_rhs(m, sys, h, u, H, U);
        for (int i = 0; i < nC; ++i) h1[i] = ssp_stage1(h[i], H[i], dt);
        for (int e = 0; e < nE; ++e) u1[e] = ssp_stage1(u[e], U[e], dt);
        or_rhs(m, sys, h1, u1, H, U);
        for (int i = 0; i < nC; ++i) h[i] = ssp2_stage2(h[i], h1[i], H[i], dt);
        for (int e = 0; e < nE; ++e) u[e] = ssp2_stage2(u[e], u1[e], U[e], dt);
    }
    free(h1); free(u1); free(H); free(U);
}

/* ------------------------------------------------------------------ LTS3 */

/* Steps 3.1.1 / 3.2.1 / 3.3.1 for LTS3:
 *   alpha_k = k/M,        alpha~_k = k^2/M^2
 *   beta_k  = (k+1)/M,    beta~_k  = k(k+2)/M^2
 *   gamma_k = (2k+1)/(2M), gamma~_k = (2k^2+2k+1)/(2M^2)
 * x = (1 - a - a~) x_old + (a - a~) x_1st + 2 a~ x_2nd. */
void or_lts3_predict_coeffs(int k, int M, int stage, double* c) {
    double a, at;
    double kk = (double)k, MM = (double)M;
    if (stage == 1) {
        a = kk / MM;
        at = kk * kk / (MM * MM);
    } else if (stage == 2) {
        a = (kk + 1.0) / MM;
        at = kk * (kk + 2.0) / (MM * MM);
    } else {
        a = (2.0 * kk + 1.0) / (2.0 * MM);
        at = (2.0 * kk * kk + 2.0 * kk + 1.0) / (2.0 * MM * MM);
    }
    c[0] = 1.0 - a - at;
    c[1] = a - at;
    c[2] = 2.0 * at;
}

/* Labels: cells 0 F\Fbar, 1 F2, 2 F1, 3 I1, 4 I2, 5 C; edges 0 F^e, 1 Fbar^e,
 * 3 I1^e, 4 I2^e, 5 C^e. */
#define C_FINE(l)  ((l) <= 2)
#define C_FBAR(l)  ((l) == 1 || (l) == 2)
#define C_I1(l)    ((l) == 3)
#define C_I(l)     ((l) == 3 || (l) == 4)
#define C_C(l)     ((l) == 5)
#define E_FINE(l)  ((l) <= 1)            /* F^e u Fbar^e (reading R1) */
#define E_FBAR(l)  ((l) == 1)

int or_lts3(const or_mesh* m, const or_system* sys, const signed char* cl,
            const signed char* el, int M, double dt, int nsteps, int step5_form,
            double* h, double* u) {
    if (M < 1) return -1;
    int nC = m->nC, nE = m->nE;
    size_t sc = (size_t)nC * sizeof(double), se = (size_t)nE * sizeof(double);
    double *h_old = xmalloc(sc), *u_old = xmalloc(se);
    double *h_1st = xmalloc(sc), *u_1st = xmalloc(se);
    double *h_2nd = xmalloc(sc), *u_2nd = xmalloc(se);
    double *h_oldk = xmalloc(sc), *u_oldk = xmalloc(se);
    double *h_1stk = xmalloc(sc), *u_1stk = xmalloc(se);
    double *h_2ndk = xmalloc(sc), *u_2ndk = xmalloc(se);
    double *H1 = xmalloc(sc), *H2 = xmalloc(sc), *H3 = xmalloc(sc);
    double *U1 = xmalloc(se), *U2 = xmalloc(se), *U3 = xmalloc(se);
    double *H = xmalloc(sc), *U = xmalloc(se);
    double dtM = dt / (double)M;
    double c[3];

    for (int n = 0; n < nsteps; ++n) {
        memcpy(h_old, h, sc); memcpy(u_old, u, se);
        /* initialisation: (h^1st,u^1st) = (h^2nd,u^2nd) = (h^old,u^old) */
        memcpy(h_1st, h_old, sc); memcpy(u_1st, u_old, se);
        memcpy(h_2nd, h_old, sc); memcpy(u_2nd, u_old, se);

        /* Step 1: first stage on Fbar u I1 u I2 u C (cells and edges). */
        or_rhs(m, sys, h_old, u_old, H, U);
        for (int i = 0; i < nC; ++i)
            if (!C_FINE(cl[i]) || C_FBAR(cl[i])) h_1st[i] = ssp_stage1(h_old[i], H[i], dt);
        for (int e = 0; e < nE; ++e)
            if (!E_FINE(el[e]) || E_FBAR(el[e])) u_1st[e] = ssp_stage1(u_old[e], U[e], dt);

        /* Step 2: second stage on I1 u I2 u C. */
        or_rhs(m, sys, h_1st, u_1st, H, U);
        for (int i = 0; i < nC; ++i)
            if (cl[i] >= 3) h_2nd[i] = ssp_stage2(h_old[i], h_1st[i], H[i], dt);
        for (int e = 0; e < nE; ++e)
            if (el[e] >= 3) u_2nd[e] = ssp_stage2(u_old[e], u_1st[e], U[e], dt);

        /* Step 3: initialisation (stage vectors start from the coarse stage
         * values everywhere, reading R4), correction terms set to zero. */
        memcpy(h_oldk, h_old, sc); memcpy(u_oldk, u_old, se);
        memcpy(h_1stk, h_1st, sc); memcpy(u_1stk, u_1st, se);
        memcpy(h_2ndk, h_2nd, sc); memcpy(u_2ndk, u_2nd, se);
        for (int i = 0; i < nC; ++i) H1[i] = H2[i] = H3[i] = 0.0;
        for (int e = 0; e < nE; ++e) U1[e] = U2[e] = U3[e] = 0.0;

        for (int k = 0; k < M; ++k) {
            /* 3.1.1 predict I1 */
            or_lts3_predict_coeffs(k, M, 1, c);
            for (int i = 0; i < nC; ++i)
                if (C_I1(cl[i])) h_oldk[i] = c[0] * h_old[i] + c[1] * h_1st[i] + c[2] * h_2nd[i];
            for (int e = 0; e < nE; ++e)
                if (el[e] == 3) u_oldk[e] = c[0] * u_old[e] + c[1] * u_1st[e] + c[2] * u_2nd[e];
            /* 3.1.2 correction terms on I1 u I2 */
            or_rhs(m, sys, h_oldk, u_oldk, H, U);
            for (int i = 0; i < nC; ++i) if (C_I(cl[i])) H1[i] = H1[i] + H[i];
            for (int e = 0; e < nE; ++e) if (el[e] == 3 || el[e] == 4) U1[e] = U1[e] + U[e];
            /* 3.1.3 fine advance */
            for (int i = 0; i < nC; ++i)
                if (C_FINE(cl[i])) h_1stk[i] = ssp_stage1(h_oldk[i], H[i], dtM);
            for (int e = 0; e < nE; ++e)
                if (E_FINE(el[e])) u_1stk[e] = ssp_stage1(u_oldk[e], U[e], dtM);

            /* 3.2.1 predict I1 */
            or_lts3_predict_coeffs(k, M, 2, c);
            for (int i = 0; i < nC; ++i)
                if (C_I1(cl[i])) h_1stk[i] = c[0] * h_old[i] + c[1] * h_1st[i] + c[2] * h_2nd[i];
            for (int e = 0; e < nE; ++e)
                if (el[e] == 3) u_1stk[e] = c[0] * u_old[e] + c[1] * u_1st[e] + c[2] * u_2nd[e];
            /* 3.2.2 */
            or_rhs(m, sys, h_1stk, u_1stk, H, U);
            for (int i = 0; i < nC; ++i) if (C_I(cl[i])) H2[i] = H2[i] + H[i];
            for (int e = 0; e < nE; ++e) if (el[e] == 3 || el[e] == 4) U2[e] = U2[e] + U[e];
            /* 3.2.3 (reading R3) */
            for (int i = 0; i < nC; ++i)
                if (C_FINE(cl[i])) h_2ndk[i] = ssp_stage2(h_oldk[i], h_1stk[i], H[i], dtM);
            for (int e = 0; e < nE; ++e)
                if (E_FINE(el[e])) u_2ndk[e] = ssp_stage2(u_oldk[e], u_1stk[e], U[e], dtM);

            /* 3.3.1 predict I1 */
            or_lts3_predict_coeffs(k, M, 3, c);
            for (int i = 0; i < nC; ++i)
                if (C_I1(cl[i])) h_2ndk[i] = c[0] * h_old[i] + c[1] * h_1st[i] + c[2] * h_2nd[i];
            for (int e = 0; e < nE; ++e)
                if (el[e] == 3) u_2ndk[e] = c[0] * u_old[e] + c[1] * u_1st[e] + c[2] * u_2nd[e];
            /* 3.3.2 */
            or_rhs(m, sys, h_2ndk, u_2ndk, H, U);
            for (int i = 0; i < nC; ++i) if (C_I(cl[i])) H3[i] = H3[i] + H[i];
            for (int e = 0; e < nE; ++e) if (el[e] == 3 || el[e] == 4) U3[e] = U3[e] + U[e];
            /* 3.3.3 (readings R2, R3) and h^{old,k+1} = h^{new} on the fine sets (R1) */
            for (int i = 0; i < nC; ++i)
                if (C_FINE(cl[i])) h_oldk[i] = ssp_stage3(h_oldk[i], h_2ndk[i], H[i], dtM);
            for (int e = 0; e < nE; ++e)
                if (E_FINE(el[e])) u_oldk[e] = ssp_stage3(u_oldk[e], u_2ndk[e], U[e], dtM);
        }

        /* Step 4: third stage on C (reading R2). */
        or_rhs(m, sys, h_2nd, u_2nd, H, U);
        for (int i = 0; i < nC; ++i)
            if (C_C(cl[i])) h[i] = ssp_stage3(h_old[i], h_2nd[i], H[i], dt);
        for (int e = 0; e < nE; ++e)
            if (el[e] == 5) u[e] = ssp_stage3(u_old[e], u_2nd[e], U[e], dt);

        /* Fine sets: the result of the last substep. */
        for (int i = 0; i < nC; ++i) if (C_FINE(cl[i])) h[i] = h_oldk[i];
        for (int e = 0; e < nE; ++e) if (E_FINE(el[e])) u[e] = u_oldk[e];

        /* Step 5: interface correction on I1 u I2. */
        for (int i = 0; i < nC; ++i) {
            if (!C_I(cl[i])) continue;
            if (step5_form == 1) {
                h[i] = h_old[i] + dtM * (H1[i] / 6.0 + H2[i] / 6.0 + 2.0 * H3[i] / 3.0);
            } else {
                double x1 = ssp_stage1(h_old[i], H1[i], dtM);
                double x2 = ssp_stage2(h_old[i], x1, H2[i], dtM);
                h[i] = ssp_stage3(h_old[i], x2, H3[i], dtM);
            }
        }
        for (int e = 0; e < nE; ++e) {
            if (!(el[e] == 3 || el[e] == 4)) continue;
            if (step5_form == 1) {
                u[e] = u_old[e] + dtM * (U1[e] / 6.0 + U2[e] / 6.0 + 2.0 * U3[e] / 3.0);
            } else {
                double x1 = ssp_stage1(u_old[e], U1[e], dtM);
                double x2 = ssp_stage2(u_old[e], x1, U2[e], dtM);
                u[e] = ssp_stage3(u_old[e], x2, U3[e], dtM);
            }
        }
    }
    free(h_old); free(u_old); free(h_1st); free(u_1st); free(h_2nd); free(u_2nd);
    free(h_oldk); free(u_oldk); free(h_1stk); free(u_1stk); free(h_2ndk); free(u_2ndk);
    free(H1); free(H2); free(H3); free(U1); free(U2); free(U3); free(H); free(U);
    return 0;
}

/* ------------------------------------------------------------------ LTS2 */

/* Steps 3.1.1 / 3.2.1 for LTS2: alpha_k = k/M, beta_k = (k+1)/M and the
 * tilde coefficients are 0, so x = (1 - a) x_old + a x_1st. */
void or_lts2_predict_coeffs(int k, int M, int stage, double* c) {
    double a = stage == 1 ? (double)k / (double)M : (double)(k + 1) / (double)M;
    c[0] = 1.0 - a;
    c[1] = a;
    c[2] = 0.0;
}

int or_lts2(const or_mesh* m, const or_system* sys, const signed char* cl,
            const signed char* el, int M, double dt, int nsteps, int step5_form,
            double* h, double* u) {
    if (M < 1) return -1;
    int nC = m->nC, nE = m->nE;
    size_t sc = (size_t)nC * sizeof(double), se = (size_t)nE * sizeof(double);
    double *h_old = xmalloc(sc), *u_old = xmalloc(se);
    double *h_1st = xmalloc(sc), *u_1st = xmalloc(se);
    double *h_2nd = xmalloc(sc), *u_2nd = xmalloc(se);
    double *h_oldk = xmalloc(sc), *u_oldk = xmalloc(se);
    double *h_1stk = xmalloc(sc), *u_1stk = xmalloc(se);
    double *H1 = xmalloc(sc), *H2 = xmalloc(sc);
    double *U1 = xmalloc(se), *U2 = xmalloc(se);
    double *H = xmalloc(sc), *U = xmalloc(se);
    double dtM = dt / (double)M;
    double c[3];

    for (int n = 0; n < nsteps; ++n) {
        memcpy(h_old, h, sc); memcpy(u_old, u, se);
        memcpy(h_1st, h_old, sc); memcpy(u_1st, u_old, se);
        memcpy(h_2nd, h_old, sc); memcpy(u_2nd, u_old, se);

        /* Step 1: first stage on I1 u I2 u C (no Fbar for LTS2). */
        or_rhs(m, sys, h_old, u_old, H, U);
        for (int i = 0; i < nC; ++i) if (cl[i] >= 3) h_1st[i] = ssp_stage1(h_old[i], H[i], dt);
        for (int e = 0; e < nE; ++e) if (el[e] >= 3) u_1st[e] = ssp_stage1(u_old[e], U[e], dt);

        /* Step 2: second stage on C only. */
        or_rhs(m, sys, h_1st, u_1st, H, U);
        for (int i = 0; i < nC; ++i) if (C_C(cl[i])) h_2nd[i] = ssp2_stage2(h_old[i], h_1st[i], H[i], dt);
        for (int e = 0; e < nE; ++e) if (el[e] == 5) u_2nd[e] = ssp2_stage2(u_old[e], u_1st[e], U[e], dt);

        /* Step 3 (reading R4: the stage vectors start from the coarse stage
         * values everywhere; two correction terms for LTS2). */
        memcpy(h_oldk, h_old, sc); memcpy(u_oldk, u_old, se);
        memcpy(h_1stk, h_1st, sc); memcpy(u_1stk, u_1st, se);
        for (int i = 0; i < nC; ++i) H1[i] = H2[i] = 0.0;
        for (int e = 0; e < nE; ++e) U1[e] = U2[e] = 0.0;

        for (int k = 0; k < M; ++k) {
            /* 3.1.1 predict I1 */
            or_lts2_predict_coeffs(k, M, 1, c);
            for (int i = 0; i < nC; ++i)
                if (C_I1(cl[i])) h_oldk[i] = c[0] * h_old[i] + c[1] * h_1st[i] + c[2] * h_2nd[i];
            for (int e = 0; e < nE; ++e)
                if (el[e] == 3) u_oldk[e] = c[0] * u_old[e] + c[1] * u_1st[e] + c[2] * u_2nd[e];
            /* 3.1.2 */
            or_rhs(m, sys, h_oldk, u_oldk, H, U);
            for (int i = 0; i < nC; ++i) if (C_I(cl[i])) H1[i] = H1[i] + H[i];
            for (int e = 0; e < nE; ++e) if (el[e] == 3 || el[e] == 4) U1[e] = U1[e] + U[e];
            /* 3.1.3 */
            for (int i = 0; i < nC; ++i)
                if (C_FINE(cl[i])) h_1stk[i] = ssp_stage1(h_oldk[i], H[i], dtM);
            for (int e = 0; e < nE; ++e)
                if (E_FINE(el[e])) u_1stk[e] = ssp_stage1(u_oldk[e], U[e], dtM);

            /* 3.2.1 predict I1 */
            or_lts2_predict_coeffs(k, M, 2, c);
            for (int i = 0; i < nC; ++i)
                if (C_I1(cl[i])) h_1stk[i] = c[0] * h_old[i] + c[1] * h_1st[i] + c[2] * h_2nd[i];
            for (int e = 0; e < nE; ++e)
                if (el[e] == 3) u_1stk[e] = c[0] * u_old[e] + c[1] * u_1st[e] + c[2] * u_2nd[e];
            /* 3.2.2 */
            or_rhs(m, sys, h_1stk, u_1stk, H, U);
            for (int i = 0; i < nC; ++i) if (C_I(cl[i])) H2[i] = H2[i] + H[i];
            for (int e = 0; e < nE; ++e) if (el[e] == 3 || el[e] == 4) U2[e] = U2[e] + U[e];
            /* 3.2.3 (reading R3); LTS2: h^new = h^2nd, then h^{old,k+1} = h^new */
            for (int i = 0; i < nC; ++i)
                if (C_FINE(cl[i])) h_oldk[i] = ssp2_stage2(h_oldk[i], h_1stk[i], H[i], dtM);
            for (int e = 0; e < nE; ++e)
                if (E_FINE(el[e])) u_oldk[e] = ssp2_stage2(u_oldk[e], u_1stk[e], U[e], dtM);
        }

        /* Step 4 (LTS2): h^new = h^2nd on C. */
        for (int i = 0; i < nC; ++i) if (C_C(cl[i])) h[i] = h_2nd[i];
        for (int e = 0; e < nE; ++e) if (el[e] == 5) u[e] = u_2nd[e];
        /* fine sets: the last substep */
        for (int i = 0; i < nC; ++i) if (C_FINE(cl[i])) h[i] = h_oldk[i];
        for (int e = 0; e < nE; ++e) if (E_FINE(el[e])) u[e] = u_oldk[e];

        /* Step 5 (theta = 1/2, 1/2, 0), printed or as the replay of the two
         * interface stages (reading R5). */
        for (int i = 0; i < nC; ++i) {
            if (!C_I(cl[i])) continue;
            if (step5_form == 1) {
                h[i] = h_old[i] + dtM * (H1[i] / 2.0 + H2[i] / 2.0);
            } else {
                double x1 = ssp_stage1(h_old[i], H1[i], dtM);
                h[i] = ssp2_stage2(h_old[i], x1, H2[i], dtM);
            }
        }
        for (int e = 0; e < nE; ++e) {
            if (!(el[e] == 3 || el[e] == 4)) continue;
            if (step5_form == 1) {
                u[e] = u_old[e] + dtM * (U1[e] / 2.0 + U2[e] / 2.0);
            } else {
                double x1 = ssp_stage1(u_old[e], U1[e], dtM);
                u[e] = ssp2_stage2(u_old[e], x1, U2[e], dtM);
            }
        }
    }
    free(h_old); free(u_old); free(h_1st); free(u_1st); free(h_2nd); free(u_2nd);
    free(h_oldk); free(u_oldk); free(h_1stk); free(u_1stk);
    free(H1); free(H2); free(U1); free(U2); free(H); free(U);
    return 0;
}

/* ---------------------------------------------- several fine regions (LTS3) */

/* Region of every cell and edge of the fine and interface sets: a walk out
 * of each region's fine cells through the non-coarse cells (labels 0..4);
 * 0 for the coarse sets.  Returns -1 if two regions' sets touch. */
int or_region_ids(const or_mesh* m, const signed char* region_of_fine, const signed char* cl,
                  const signed char* el, signed char* creg, signed char* ereg) {
    int nC = m->nC, nE = m->nE, bad = 0;
    int* queue = (int*)xmalloc((size_t)nC * sizeof(int));
    int head = 0, tail = 0;
    for (int i = 0; i < nC; ++i) {
        creg[i] = 0;
        if (cl[i] <= 2 && region_of_fine[i] > 0) {
            creg[i] = region_of_fine[i];
            queue[tail++] = i;
        }
    }
    while (head < tail) {
        int i = queue[head++];
        for (int j = 0; j < m->nEoC[i]; ++j) {
            int e = m->EoC[(size_t)i * m->maxE + j];
            int nb = m->CoE[2 * e] == i ? m->CoE[2 * e + 1] : m->CoE[2 * e];
            if (cl[nb] == 5) continue;
            if (creg[nb] == 0) {
                creg[nb] = creg[i];
                queue[tail++] = nb;
            } else if (creg[nb] != creg[i]) {
                bad = 1;
            }
        }
    }
    for (int e = 0; e < nE; ++e) {
        int a = m->CoE[2 * e], b = m->CoE[2 * e + 1];
        ereg[e] = el[e] == 5 ? 0 : (cl[a] <= cl[b] ? creg[a] : creg[b]);
    }
    free(queue);
    return bad ? -1 : 0;
}

int or_lts3_multi(const or_mesh* m, const or_system* sys, const signed char* cl,
                  const signed char* el, const signed char* creg, const signed char* ereg,
                  int nreg, const int* Ms, double dt, int nsteps, int step5_form, double* h,
                  double* u) {
    for (int r = 0; r < nreg; ++r)
        if (Ms[r] < 1) return -1;
    int nC = m->nC, nE = m->nE;
    size_t sc = (size_t)nC * sizeof(double), se = (size_t)nE * sizeof(double);
    double *h_old = xmalloc(sc), *u_old = xmalloc(se);
    double *h_1st = xmalloc(sc), *u_1st = xmalloc(se);
    double *h_2nd = xmalloc(sc), *u_2nd = xmalloc(se);
    double *h_oldk = xmalloc(sc), *u_oldk = xmalloc(se);
    double *h_1stk = xmalloc(sc), *u_1stk = xmalloc(se);
    double *h_2ndk = xmalloc(sc), *u_2ndk = xmalloc(se);
    double *H1 = xmalloc(sc), *H2 = xmalloc(sc), *H3 = xmalloc(sc);
    double *U1 = xmalloc(se), *U2 = xmalloc(se), *U3 = xmalloc(se);
    double *H = xmalloc(sc), *U = xmalloc(se);
    double c[3];

    for (int n = 0; n < nsteps; ++n) {
        memcpy(h_old, h, sc); memcpy(u_old, u, se);
        memcpy(h_1st, h_old, sc); memcpy(u_1st, u_old, se);
        memcpy(h_2nd, h_old, sc); memcpy(u_2nd, u_old, se);
        /* Steps 1 and 2 on the union of the sets, as for one region */
        or_rhs(m, sys, h_old, u_old, H, U);
        for (int i = 0; i < nC; ++i)
            if (!C_FINE(cl[i]) || C_FBAR(cl[i])) h_1st[i] = ssp_stage1(h_old[i], H[i], dt);
        for (int e = 0; e < nE; ++e)
            if (!E_FINE(el[e]) || E_FBAR(el[e])) u_1st[e] = ssp_stage1(u_old[e], U[e], dt);
        or_rhs(m, sys, h_1st, u_1st, H, U);
        for (int i = 0; i < nC; ++i)
            if (cl[i] >= 3) h_2nd[i] = ssp_stage2(h_old[i], h_1st[i], H[i], dt);
        for (int e = 0; e < nE; ++e)
            if (el[e] >= 3) u_2nd[e] = ssp_stage2(u_old[e], u_1st[e], U[e], dt);
        memcpy(h_oldk, h_old, sc); memcpy(u_oldk, u_old, se);
        memcpy(h_1stk, h_1st, sc); memcpy(u_1stk, u_1st, se);
        memcpy(h_2ndk, h_2nd, sc); memcpy(u_2ndk, u_2nd, se);
        for (int i = 0; i < nC; ++i) H1[i] = H2[i] = H3[i] = 0.0;
        for (int e = 0; e < nE; ++e) U1[e] = U2[e] = U3[e] = 0.0;

        /* Step 3 for each region with its own M (the regions' right-hand sides
         * read disjoint neighbourhoods, so their order does not matter) */
        for (int r = 1; r <= nreg; ++r) {
            const int M = Ms[r - 1];
            const double dtM = dt / (double)M;
#define IN_R(i) (creg[i] == r)
#define EN_R(e) (ereg[e] == r)
            for (int k = 0; k < M; ++k) {
                or_lts3_predict_coeffs(k, M, 1, c);
                for (int i = 0; i < nC; ++i)
                    if (IN_R(i) && C_I1(cl[i])) h_oldk[i] = c[0] * h_old[i] + c[1] * h_1st[i] + c[2] * h_2nd[i];
                for (int e = 0; e < nE; ++e)
                    if (EN_R(e) && el[e] == 3) u_oldk[e] = c[0] * u_old[e] + c[1] * u_1st[e] + c[2] * u_2nd[e];
                or_rhs(m, sys, h_oldk, u_oldk, H, U);
                for (int i = 0; i < nC; ++i) if (IN_R(i) && C_I(cl[i])) H1[i] = H1[i] + H[i];
                for (int e = 0; e < nE; ++e) if (EN_R(e) && (el[e] == 3 || el[e] == 4)) U1[e] = U1[e] + U[e];
                for (int i = 0; i < nC; ++i)
                    if (IN_R(i) && C_FINE(cl[i])) h_1stk[i] = ssp_stage1(h_oldk[i], H[i], dtM);
                for (int e = 0; e < nE; ++e)
                    if (EN_R(e) && E_FINE(el[e])) u_1stk[e] = ssp_stage1(u_oldk[e], U[e], dtM);

                or_lts3_predict_coeffs(k, M, 2, c);
                for (int i = 0; i < nC; ++i)
                    if (IN_R(i) && C_I1(cl[i])) h_1stk[i] = c[0] * h_old[i] + c[1] * h_1st[i] + c[2] * h_2nd[i];
                for (int e = 0; e < nE; ++e)
                    if (EN_R(e) && el[e] == 3) u_1stk[e] = c[0] * u_old[e] + c[1] * u_1st[e] + c[2] * u_2nd[e];
                or_rhs(m, sys, h_1stk, u_1stk, H, U);
                for (int i = 0; i < nC; ++i) if (IN_R(i) && C_I(cl[i])) H2[i] = H2[i] + H[i];
                for (int e = 0; e < nE; ++e) if (EN_R(e) && (el[e] == 3 || el[e] == 4)) U2[e] = U2[e] + U[e];
                for (int i = 0; i < nC; ++i)
                    if (IN_R(i) && C_FINE(cl[i])) h_2ndk[i] = ssp_stage2(h_oldk[i], h_1stk[i], H[i], dtM);
                for (int e = 0; e < nE; ++e)
                    if (EN_R(e) && E_FINE(el[e])) u_2ndk[e] = ssp_stage2(u_oldk[e], u_1stk[e], U[e], dtM);

                or_lts3_predict_coeffs(k, M, 3, c);
                for (int i = 0; i < nC; ++i)
                    if (IN_R(i) && C_I1(cl[i])) h_2ndk[i] = c[0] * h_old[i] + c[1] * h_1st[i] + c[2] * h_2nd[i];
                for (int e = 0; e < nE; ++e)
                    if (EN_R(e) && el[e] == 3) u_2ndk[e] = c[0] * u_old[e] + c[1] * u_1st[e] + c[2] * u_2nd[e];
                or_rhs(m, sys, h_2ndk, u_2ndk, H, U);
                for (int i = 0; i < nC; ++i) if (IN_R(i) && C_I(cl[i])) H3[i] = H3[i] + H[i];
                for (int e = 0; e < nE; ++e) if (EN_R(e) && (el[e] == 3 || el[e] == 4)) U3[e] = U3[e] + U[e];
                for (int i = 0; i < nC; ++i)
                    if (IN_R(i) && C_FINE(cl[i])) h_oldk[i] = ssp_stage3(h_oldk[i], h_2ndk[i], H[i], dtM);
                for (int e = 0; e < nE; ++e)
                    if (EN_R(e) && E_FINE(el[e])) u_oldk[e] = ssp_stage3(u_oldk[e], u_2ndk[e], U[e], dtM);
            }
#undef IN_R
#undef EN_R
        }

        /* Step 4 on C */
        or_rhs(m, sys, h_2nd, u_2nd, H, U);
        for (int i = 0; i < nC; ++i)
            if (C_C(cl[i])) h[i] = ssp_stage3(h_old[i], h_2nd[i], H[i], dt);
        for (int e = 0; e < nE; ++e)
            if (el[e] == 5) u[e] = ssp_stage3(u_old[e], u_2nd[e], U[e], dt);
        for (int i = 0; i < nC; ++i) if (C_FINE(cl[i])) h[i] = h_oldk[i];
        for (int e = 0; e < nE; ++e) if (E_FINE(el[e])) u[e] = u_oldk[e];

        /* Step 5 on each region's interface with its own dt/M */
        for (int i = 0; i < nC; ++i) {
            if (!C_I(cl[i]) || creg[i] < 1) continue;
            const double dtM = dt / (double)Ms[creg[i] - 1];
            if (step5_form == 1) {
                h[i] = h_old[i] + dtM * (H1[i] / 6.0 + H2[i] / 6.0 + 2.0 * H3[i] / 3.0);
            } else {
                double x1 = ssp_stage1(h_old[i], H1[i], dtM);
                double x2 = ssp_stage2(h_old[i], x1, H2[i], dtM);
                h[i] = ssp_stage3(h_old[i], x2, H3[i], dtM);
            }
        }
        for (int e = 0; e < nE; ++e) {
            if (!(el[e] == 3 || el[e] == 4) || ereg[e] < 1) continue;
            const double dtM = dt / (double)Ms[ereg[e] - 1];
            if (step5_form == 1) {
                u[e] = u_old[e] + dtM * (U1[e] / 6.0 + U2[e] / 6.0 + 2.0 * U3[e] / 3.0);
            } else {
                double x1 = ssp_stage1(u_old[e], U1[e], dtM);
                double x2 = ssp_stage2(u_old[e], x1, U2[e], dtM);
                u[e] = ssp_stage3(u_old[e], x2, U3[e], dtM);
            }
        }
    }
    free(h_old); free(u_old); free(h_1st); free(u_1st); free(h_2nd); free(u_2nd);
    free(h_oldk); free(u_oldk); free(h_1stk); free(u_1stk); free(h_2ndk); free(u_2ndk);
    free(H1); free(H2); free(H3); free(U1); free(U2); free(U3); free(H); free(U);
    return 0;
}

/* ------------------------------------------------------------ diagnostics */

double or_mass(const or_mesh* m, const double* h) {
    double s = 0.0;
    for (int i = 0; i < m->nC; ++i) s += m->A[i] * h[i];
    return s;
}

double or_energy(const or_mesh* m, double g, const double* h, const double* u) {
    double* K = (double*)xmalloc((size_t)m->nC * sizeof(double));
    or_kinetic(m, u, K);
    double s = 0.0;
    for (int i = 0; i < m->nC; ++i) s += m->A[i] * h[i] * (K[i] + g * (0.5 * h[i] + m->b[i]));
    free(K);
    return s;
}

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
