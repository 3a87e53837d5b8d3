/*
 * oracle.h -- plain FP64 CPU oracle for the TRiSK shallow-water right-hand side
 * and the SSP-RK3 / LTS3 time integrators of Capodaglio & Petersen,
 * "Local time stepping for the shallow water equations in MPAS"
 * (arXiv:2106.07154).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library includes this
 * header or links this code; only the tests, the smoke check and the CPU
 * baseline of the benchmark load it.  It shares no code, header, table or
 * helper with the GPU path.
 *
 * Mesh convention (input, MPAS-style, 0-based):
 *   cellsOnEdge[2e+0], cellsOnEdge[2e+1] : the two cells of edge e; the normal
 *       n_e points out of cellsOnEdge[2e+0] (so n_{e,i} = +1 for that cell).
 *   verticesOnEdge[2e+0], [2e+1]         : the two end vertices of e;
 *       verticesOnEdge[2e+1] lies in the direction k x n_e (t_{e,v} = +1).
 *   edgesOnCell[i*maxEdges + j], j < nEdgesOnCell[i] : edges of cell i, in
 *       order around the cell (either sense; Appendix B lets the weight
 *       path run clockwise or counter-clockwise).
 *   cellsOnVertex[3v+k], edgesOnVertex[3v+k], kiteAreasOnVertex[3v+k]: the
 *       kite area A_{i,v} of cell cellsOnVertex[3v+k] at vertex v.
 *   l_e = dvEdge (primal Voronoi edge length), d_e = dcEdge (dual edge,
 *   cell-to-cell distance), A_i = areaCell, A_v = areaTriangle.
 *
 * Parity status: every function here is pinned by the CPU tests (closed
 * forms, invariants, brute force, the M = 1 identity of the paper's Remark
 * in Section 2.2, and for the energy of reading R8 a closed form and its
 * conservation by the semi-discrete system of Eq. (1)).  The paper prints no
 * solution values, so no pin compares against a printed number.
 */
#ifndef LTS_ORACLE_H
#define LTS_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct or_mesh or_mesh;

/* Copies the arrays; returns NULL on inconsistent input. */
or_mesh* or_mesh_new(int nCells, int nEdges, int nVertices, int maxEdges,
                     const int* nEdgesOnCell, const int* edgesOnCell,
                     const int* cellsOnEdge, const int* verticesOnEdge,
                     const int* edgesOnVertex, const int* cellsOnVertex,
                     const double* areaCell, const double* areaTriangle,
                     const double* kiteAreasOnVertex, const double* dcEdge,
                     const double* dvEdge, const double* fVertex,
                     const double* bottom);
void or_mesh_free(or_mesh* m);

/* EE(e) and w_{e,e'} of Appendix B, Eq. (weights).  eoe/woe are
 * [nEdges * 2*maxEdges]; neoe[nEdges] receives |EE(e)|. */
void or_weights(const or_mesh* m, int* neoe, int* eoe, double* woe);

/* Individual TRiSK operators of Appendix B. */
void or_divergence(const or_mesh* m, const double* F, double* div);      /* [div F]_i       */
void or_gradient(const or_mesh* m, const double* phi, double* grad);     /* [grad phi]_e    */
void or_vorticity(const or_mesh* m, const double* u, double* zeta);      /* zeta_v          */
void or_kinetic(const or_mesh* m, const double* u, double* K);           /* K_i             */
void or_thickness_flux(const or_mesh* m, const double* h, const double* u, double* F);
void or_pv_vertex(const or_mesh* m, const double* h, const double* u, double* q);
void or_pv_flux(const or_mesh* m, const double* F, const double* qe, double* pv); /* F_e^perp [q]_{v->e} */
void or_tangential(const or_mesh* m, const double* F, double* Fperp);   /* F_e^perp        */

/* Eq. (1): H_i(h,u) and U_e(h,u) evaluated on the whole mesh. */
void or_rhs_swe(const or_mesh* m, double g, const double* h, const double* u,
                double* H, double* U);

/* Region labels of Eqs. (3)-(5).
 * cell_label: 0 F \ Fbar, 1 F2, 2 F1, 3 I1, 4 I2, 5 C  (Fbar = F1 u F2)
 * edge_label: 0 F^e, 1 Fbar^e, 3 I1^e, 4 I2^e, 5 C^e                   */
int or_regions(const or_mesh* m, const signed char* fine_mask,
               signed char* cell_label, signed char* edge_label);
/* The same with interfaces L cells thick: I1 = the non-fine cells reached
 * from F by 1..L edge crossings, I2 = those reached by L+1..2L (the thick
 * interface layers of the speed-up runs of Section 3; L = 1 is Eq. 3).
 * F1, F2 and the edge sets follow Eqs. (4)-(5) unchanged.  Returns -1 for
 * L < 1. */
int or_regions_layers(const or_mesh* m, const signed char* fine_mask, int L,
                      signed char* cell_label, signed char* edge_label);

/* Prediction coefficients of Steps 3.1.1 / 3.2.1 / 3.3.1 (LTS3):
 * x = c[0]*x_old + c[1]*x_1st + c[2]*x_2nd.  stage = 1, 2, 3. */
void or_lts3_predict_coeffs(int k, int M, int stage, double* c);

/* Systems the integrators can advance. */
enum { OR_SYS_SWE = 0, OR_SYS_LINEAR = 1 };
/* OR_SYS_LINEAR: decoupled linear test system H_i = lam_c[i] h_i,
 * U_e = lam_e[e] u_e (used by the closed-form pins). */

typedef struct {
    int kind;
    double g;
    const double* lam_c;
    const double* lam_e;
} or_system;

void or_rhs(const or_mesh* m, const or_system* sys, const double* h, const double* u,
            double* H, double* U);

/* Algorithm 2.1 (SSPRK3), n steps of size dt, (h,u) advanced in place. */
void or_ssprk3(const or_mesh* m, const or_system* sys, double dt, int nsteps,
               double* h, double* u);
/* Algorithm 2.1 (SSPRK2: omega = 1/2, 1/2, 1/2), n steps of size dt. */
void or_ssprk2(const or_mesh* m, const or_system* sys, double dt, int nsteps,
               double* h, double* u);
/* Classical RK4 (reference-solution generator, Section 3.2). */
void or_rk4(const or_mesh* m, const or_system* sys, double dt, int nsteps,
            double* h, double* u);
/* Algorithm 2.2 (LTS3), n coarse steps of size dt with M fine substeps.
 * step5_form: 0 = Shu-Osher replay of the three interface stages
 *             (algebraically identical to Step 5), 1 = Step 5 as printed. */
int or_lts3(const or_mesh* m, const or_system* sys, const signed char* cell_label,
            const signed char* edge_label, int M, double dt, int nsteps,
            int step5_form, double* h, double* u);

/* Algorithm 2.2 (LTS2 branches): Step 1 on I1 u I2 u C, Step 2 on C,
 * Step 3 with two stages per substep (alpha_k = k/M, beta_k = (k+1)/M, no
 * tilde terms), Step 4 h^new = h^2nd on C, Step 5 with theta = 1/2, 1/2.
 * step5_form as for or_lts3. */
int or_lts2(const or_mesh* m, const or_system* sys, const signed char* cell_label,
            const signed char* edge_label, int M, double dt, int nsteps,
            int step5_form, double* h, double* u);
/* Steps 3.1.1 / 3.2.1 coefficients for LTS2 (stage 1 or 2), as for LTS3. */
void or_lts2_predict_coeffs(int k, int M, int stage, double* c);

/* Several disjoint fine regions r = 1..nreg, each with its own M_r, sharing
 * the coarse step (the regions of the Remark in Section 2.3, not nested):
 * Steps 1, 2 and 4 of Algorithm 2.2 on the union of the sets, Step 3 and
 * Step 5 per region with M_r on its own F, I1, I2.  Labels come from
 * or_regions on the union of the regions' cells; creg/ereg from
 * or_region_ids (0 = coarse).  The regions' sets must not touch. */
int or_region_ids(const or_mesh* m, const signed char* region_of_fine, const signed char* cell_label,
                  const signed char* edge_label, signed char* creg, signed char* ereg);
int or_lts3_multi(const or_mesh* m, const or_system* sys, const signed char* cell_label,
                  const signed char* edge_label, const signed char* creg, const signed char* ereg,
                  int nreg, const int* M, double dt, int nsteps, int step5_form, double* h,
                  double* u);

/* Diagnostics: mass sum_i A_i h_i and energy sum_i A_i h_i (K_i + g(h_i/2 + b_i)). */
double or_mass(const or_mesh* m, const double* h);
double or_energy(const or_mesh* m, double g, const double* h, const double* u);

int or_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
