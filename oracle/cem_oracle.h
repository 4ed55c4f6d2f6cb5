/*
 * cem_oracle.h -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, single-threaded FP64 CPU restatement of the explicit
 * MCT-2D-CEM time step on a structured bilinear-quadrilateral (Q4) mesh.
 * It is the parity judge of the CUDA library: only tests, the smoke check
 * and the benchmark's CPU-baseline leg may load it.  It shares no code,
 * header, table or constant with the CUDA path.
 *
 * Conventions (identical in meaning, not in code, to the library's):
 *   node (i,j), 0<=i<=nx, 0<=j<=ny:   id = j*(nx+1)+i,  X = (i*hx, j*hy)
 *   element (i,j), 0<=i<nx, 0<=j<ny:  id = j*nx+i
 *   element local nodes (CCW): 0:(i,j) 1:(i+1,j) 2:(i+1,j+1) 3:(i,j+1)
 *   element local edges: 0 bottom, 1 right, 2 top, 3 left; edge k joins
 *   local nodes k and (k+1)%4; its quadrature point is its midpoint.
 *   edge ids: horizontal edge (i,j) [nodes (i,j)-(i+1,j)] = j*nx+i,
 *   0<=j<=ny; vertical edge (i,j) [nodes (i,j)-(i,j+1)] =
 *   nx*(ny+1) + j*(nx+1)+i, 0<=j<ny.
 *   Nodes [0,nn) are real; phantom nodes follow, in creation order.
 */
#ifndef CEM_ORACLE_H
#define CEM_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_sim orc_sim;

enum { ORC_OK = 0, ORC_ERR_ARG = -1, ORC_ERR_CAPACITY = -3, ORC_ERR_STATE = -6 };
enum { ORC_TRACTION = 0, ORC_PRESSURE = 1, ORC_VELOCITY = 2 };
enum { ORC_LAW_CONST = 0, ORC_LAW_RAMP = 1, ORC_LAW_RAMP_EXP = 2 };
enum { ORC_SCOPE_NBHD = 0, ORC_SCOPE_GLOBAL = 1, ORC_SCOPE_TIPS = 2 };
enum { ORC_GAMMA_LITERAL = 0, ORC_GAMMA_RATIO = 1 };

orc_sim *orc_create(int nx, int ny, double hx, double hy,
                    const unsigned char *active, int phantom_cap, int crack_cap);
void orc_destroy(orc_sim *s);
const char *orc_error(const orc_sim *s);

int orc_set_material(orc_sim *s, double E, double nu, double rho,
                     const float *gc, double gc_uniform, int plane_strain,
                     double gamma, int gamma_mode, int scope);
/* dt = dt_factor * min(hx,hy) / c_d, unless dt_explicit > 0. */
int orc_set_dt(orc_sim *s, double dt_factor, double dt_explicit);
double orc_dt(const orc_sim *s);
int orc_add_bc(orc_sim *s, int kind, int n, const int *items, int comp_mask,
               int law, double a0, double t0, double tau);
int orc_precrack(orc_sim *s, int n, const int *triples);
/* Sets u and v of all nodes (real, then phantom) before the first step;
 * any pointer may be NULL. */
int orc_set_state(orc_sim *s, const double *ux, const double *uy,
                  const double *vx, const double *vy);
int orc_set_energy_every(orc_sim *s, int K);
int orc_step(orc_sim *s, int nsteps);

/* counts: nn, ne, nedge, n_phantom, n_crack, step, n_surface, n_tips, n_energy */
void orc_counts(const orc_sim *s, long out[9]);
int orc_get_nodes(const orc_sim *s, double *ux, double *uy, double *vx,
                  double *vy, double *m);
int orc_get_phantoms(const orc_sim *s, int *owner, int *creator_e,
                     int *creator_a, int *nuser, int *users /* 12 each */);
int orc_get_cracks(const orc_sim *s, int *elem, int *ka, int *kb, int *step,
                   double *ud, int *nodes /* 8 each */);
int orc_get_surface(const orc_sim *s, int *edge, int *ahead, int *is_tip);
int orc_get_energy(const orc_sim *s, double *rec /* 7 each */);
int orc_internal_force(orc_sim *s, double *fx, double *fy);
int orc_eval_surface(orc_sim *s, int *edge, int *ahead, int *k0, double *G4,
                     int *prop_k);
int orc_apply_proposals(orc_sim *s, int n, const int *edge, const int *elem,
                        const int *k, const double *G);
int orc_strain_energy(orc_sim *s, double *se);
/* mean stress of each element (see the definition in cem_oracle.c) */
int orc_element_stress(orc_sim *s, double *sxx, double *syy, double *sxy);

#ifdef __cplusplus
}
#endif
#endif
