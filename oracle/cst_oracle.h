/*
 * cst_oracle.h -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, single-threaded FP64 CPU restatement of the explicit ES-FEM
 * step on an unstructured mesh of constant-strain triangles (CST), the
 * paper's own element (Sec. 2.1, Eqs. 1, 3 and 5).  Only tests may load it;
 * it shares no code, header or table with the CUDA library.
 *
 * Conventions (identical in meaning, not in code, to the library's):
 *   nodes 0..nn-1 at X[2N], X[2N+1]; element e has nodes conn[3e..3e+2],
 *   counter-clockwise; its local edge k joins local nodes k and (k+1)%3.
 *   Edges are the distinct node pairs {a, b} of the elements, numbered in
 *   increasing (min(a,b), max(a,b)); an edge has one element (boundary) or
 *   two (interior), listed in increasing element id.
 * No cracking: the triangles stay intact.
 */
#ifndef CST_ORACLE_H
#define CST_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

typedef struct ocst ocst;

/* Returns NULL on bad input (then ocst_create_error() says why). */
ocst *ocst_create(int nn, int ne, const double *X, const int *conn);
const char *ocst_create_error(void);
void ocst_destroy(ocst *s);
const char *ocst_error(const ocst *s);

int ocst_n_edges(const ocst *s);
/* edge g joins nodes n1[g] < n2[g]; its elements e1[g] < e2[g] (-1: none) */
int ocst_edges(const ocst *s, int *n1, int *n2, int *e1, int *e2);

int ocst_set_material(ocst *s, double E, double nu, double rho, int plane_strain);
/* critical energy release rate per element (gc NULL: gc_uniform) and the
 * split ratio of the CST decision rule (gamma_mode 0: G_p > gamma (G_p - G_q),
 * 1: G_p > gamma G_q) */
int ocst_set_fracture(ocst *s, const float *gc, double gc_uniform, double gamma, int gamma_mode);
/* dt = dt_factor * h_min / c_d, h_min the smallest element altitude
 * (2 A / longest edge), unless dt_explicit > 0. */
int ocst_set_dt(ocst *s, double dt_factor, double dt_explicit);
double ocst_dt(const ocst *s);
/* kind 0 traction / 1 pressure: items are boundary edge ids; kind 2
 * velocity: items are node ids.  law 0 constant, 1 ramp, 2 ramp-exp. */
int ocst_add_bc(ocst *s, int kind, int n, const int *items, int comp_mask, int law, double a0,
                double t0, double tau);
int ocst_set_state(ocst *s, const double *ux, const double *uy, const double *vx,
                   const double *vy);
int ocst_set_energy_every(ocst *s, int K);
int ocst_step(ocst *s, int nsteps);

int ocst_get_nodes(const ocst *s, double *ux, double *uy, double *vx, double *vy, double *m);
/* records of (step, t, KE, SE, W_ext, W_dir, U_d = 0), 7 doubles each */
int ocst_n_energy(const ocst *s);
int ocst_get_energy(const ocst *s, double *rec);
int ocst_internal_force(ocst *s, double *fx, double *fy);
int ocst_strain_energy(ocst *s, double *se);
/* Crack evaluation at n surface points (Sec. 2.2, CST): point q is edge
 * edge[q] of its intact element elem[q] (the element ahead).  G[2q + j]
 * is the energy release rate of the path from the point to the midpoint of
 * the element's j-th other edge (its local edges k0+1, k0+2 mod 3, k0 the
 * point's own); choice[q] the local edge of the chosen path, -1 for none. */
int ocst_eval_surface(ocst *s, int n, const int *edge, const int *elem, double *G, int *choice);

#ifdef __cplusplus
}
#endif
#endif
