/*
 * cem_oracle.c -- TEST INFRASTRUCTURE ONLY (see cem_oracle.h).
 *
 * A plain FP64 restatement of one explicit MCT-2D-CEM time step, written for
 * a reader who checks it against the paper by eye:
 *
 *   ES-FEM on Q4 elements (paper Sec. 2.1): the quadrature points are the
 *   edge midpoints; the strain at an edge point shared by two elements is the
 *   area-weighted average of the two elements' B*u there (Eqs. 1, 2, 4), and
 *   each element j receives B_j^T sigma * A_j/4 from each of its edge points
 *   (Eq. 6).  Plane Cauchy stress sigma = D eps.
 *
 *   Energy release rate of a candidate path G0->Gk (Sec. 2.2, the unnumbered
 *   release-rate equation): G = delta_d . sigma_perp(Gk) / 2 with
 *   delta_d = (u_N2 - u_N1) H(|x_N2-x_N1| / |X_N2-X_N1| - 1); Q4 cracking
 *   conditions with the split ratio gamma (Sec. 2.2, Fig. 2-3 list).
 *
 *   Multiple Crack-tips Tracking (Sec. 3): all edge points on free surfaces
 *   are candidates; those above G_c propose; the largest wins.
 *
 * Readings where the paper is silent (integrator, mass, split mechanics,
 * normal orientation, selection scope, dissipated energy) are the ones listed
 * in the design notes: central differences with half-step velocities,
 * row-sum lumped mass, phantom-node split pieces with area fractions, ES-FEM
 * smoothing switched off on every edge that touches a cracked element,
 * neighbourhood-maximum selection, U_d = sum G_c * segment length.
 *
 * Build with -O2 -ffp-contract=off: every a*b+c below is two roundings.
 */
#include "cem_oracle.h"

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

enum { ST_OUT = 0, ST_INTACT = 1, ST_CRACKED = 2 };

typedef struct {
  int elem;
  int ka, kb;      /* cut local edges: entry (surface point) and exit */
  int side[4];     /* piece (0/1) that holds local node a as a real node */
  int node[2][4];  /* node ids used by each piece (real or phantom) */
  double alpha[2]; /* area fraction of each piece */
  double Ap[2];    /* area of each piece */
  double ud;       /* dissipated energy of this split (0 for a pre-crack) */
  int step;        /* step at which the split happened (-1: pre-crack) */
} orc_crack;

typedef struct {
  int owner;       /* real node it duplicates */
  int creator_e, creator_a;
  int nuser;
  int ue[4], up[4], ua[4]; /* users: element, piece, local node; sorted by element */
} orc_phantom;

struct orc_sim {
  int nx, ny;
  double hx, hy, A;
  int nn, ne, nh, ned;
  unsigned char *active;
  /* material */
  int mat_set, plane_strain, gamma_mode, scope;
  double E, nu, rho, D11, D12, D33, gamma;
  float *gc;
  double dt;
  int dt_set;
  /* loads */
  double *Fx, *Fy;
  unsigned char *lflag;
  int neu_set, neu_law;
  double neu_t0, neu_tau;
  unsigned char *dmask;
  double *Vx, *Vy;
  int dir_set, dir_law;
  double dir_t0, dir_tau;
  /* nodes: real then phantom */
  int ncap;
  double *ux, *uy, *vx, *vy, *m, *minv, *Wn, *Wd;
  /* cracks and phantoms */
  int *crack_of;
  orc_crack *cr;
  int ncr, crcap;
  orc_phantom *ph;
  int nph, phcap;
  /* time and energy */
  int step, energy_every;
  double *erec;
  int nrec, reccap;
  /* per-step scratch */
  double *eps_own; /* ne*4*3: element's own B*u at its edge points */
  double *eps;     /* ne*4*3: strain used by an intact element at edge k */
  double *sig;     /* ne*4*3: stress used by an intact element at edge k */
  double *fe;      /* ne*8 */
  double *peps, *psig, *pf; /* crcap*2*4*3, crcap*2*4*3, crcap*2*8 */
  double *fx, *fy;
  char err[256];
};

/* ------------------------------------------------------------------ utils */

static int fail(orc_sim *s, int code, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(s->err, sizeof s->err, fmt, ap);
  va_end(ap);
  return code;
}

const char *orc_error(const orc_sim *s) { return s ? s->err : "null sim"; }

static void *zalloc(size_t n) {
  void *p = calloc(n ? n : 1, 1);
  return p;
}

/* Natural coordinates of the Q4 nodes and of the edge midpoints. */
static const double XI_N[4] = {-1.0, 1.0, 1.0, -1.0};
static const double ETA_N[4] = {-1.0, -1.0, 1.0, 1.0};
static const double XI_G[4] = {0.0, 1.0, 0.0, -1.0};
static const double ETA_G[4] = {-1.0, 0.0, 1.0, 0.0};

/* Derivatives of the bilinear shape function N_a = (1+xi_a xi)(1+eta_a eta)/4
 * of a rectangle hx*hy, evaluated at the midpoint of local edge k
 * (Eq. 4 evaluated at the edge quadrature points). */
static double dNdx(const orc_sim *s, int k, int a) {
  return XI_N[a] * (1.0 + ETA_N[a] * ETA_G[k]) / (2.0 * s->hx);
}
static double dNdy(const orc_sim *s, int k, int a) {
  return ETA_N[a] * (1.0 + XI_N[a] * XI_G[k]) / (2.0 * s->hy);
}

static void elem_nodes(const orc_sim *s, int e, int n[4]) {
  int i = e % s->nx, j = e / s->nx, r = s->nx + 1;
  n[0] = j * r + i;
  n[1] = j * r + i + 1;
  n[2] = (j + 1) * r + i + 1;
  n[3] = (j + 1) * r + i;
}

static int elem_neighbor(const orc_sim *s, int e, int k) {
  int i = e % s->nx, j = e / s->nx;
  switch (k) {
  case 0: return j > 0 ? e - s->nx : -1;
  case 1: return i < s->nx - 1 ? e + 1 : -1;
  case 2: return j < s->ny - 1 ? e + s->nx : -1;
  default: return i > 0 ? e - 1 : -1;
  }
}

static int elem_edge_id(const orc_sim *s, int e, int k) {
  int i = e % s->nx, j = e / s->nx;
  switch (k) {
  case 0: return j * s->nx + i;
  case 1: return s->nh + j * (s->nx + 1) + i + 1;
  case 2: return (j + 1) * s->nx + i;
  default: return s->nh + j * (s->nx + 1) + i;
  }
}

static int elem_status(const orc_sim *s, int e) {
  if (e < 0 || !s->active[e]) return ST_OUT;
  return s->crack_of[e] >= 0 ? ST_CRACKED : ST_INTACT;
}

/* The two elements beside edge g: lo = below/left (its local edge 2/1),
 * hi = above/right (its local edge 0/3); -1 where there is none. */
static void edge_sides(const orc_sim *s, int g, int *lo, int *klo, int *hi,
                       int *khi) {
  if (g < s->nh) {
    int j = g / s->nx, i = g % s->nx;
    *lo = j > 0 ? (j - 1) * s->nx + i : -1;
    *klo = 2;
    *hi = j < s->ny ? j * s->nx + i : -1;
    *khi = 0;
  } else {
    int gg = g - s->nh, j = gg / (s->nx + 1), i = gg % (s->nx + 1);
    *lo = i > 0 ? j * s->nx + i - 1 : -1;
    *klo = 1;
    *hi = i < s->nx ? j * s->nx + i : -1;
    *khi = 3;
  }
}

static double law_eval(int law, double t, double t0, double tau) {
  if (law == ORC_LAW_CONST) return 1.0;
  if (t <= t0) return t / t0;
  if (law == ORC_LAW_RAMP) return 1.0;
  return exp(-(t - t0) / tau);
}

/* ------------------------------------------------------------- lifecycle */

orc_sim *orc_create(int nx, int ny, double hx, double hy,
                    const unsigned char *active, int phantom_cap, int crack_cap) {
  if (nx < 1 || ny < 1 || !(hx > 0) || !(hy > 0) || phantom_cap < 0 || crack_cap < 0)
    return NULL;
  orc_sim *s = (orc_sim *)zalloc(sizeof *s);
  s->nx = nx; s->ny = ny; s->hx = hx; s->hy = hy; s->A = hx * hy;
  s->nn = (nx + 1) * (ny + 1);
  s->ne = nx * ny;
  s->nh = nx * (ny + 1);
  s->ned = s->nh + (nx + 1) * ny;
  s->active = (unsigned char *)zalloc(s->ne);
  for (int e = 0; e < s->ne; ++e) s->active[e] = active ? (active[e] != 0) : 1;
  s->phcap = phantom_cap;
  s->crcap = crack_cap;
  s->ncap = s->nn + phantom_cap;
  size_t nc = (size_t)s->ncap;
  s->ux = zalloc(nc * 8); s->uy = zalloc(nc * 8);
  s->vx = zalloc(nc * 8); s->vy = zalloc(nc * 8);
  s->m = zalloc(nc * 8); s->minv = zalloc(nc * 8);
  s->Wn = zalloc(nc * 8); s->Wd = zalloc(nc * 8);
  s->fx = zalloc(nc * 8); s->fy = zalloc(nc * 8);
  s->Fx = zalloc((size_t)s->nn * 8); s->Fy = zalloc((size_t)s->nn * 8);
  s->Vx = zalloc((size_t)s->nn * 8); s->Vy = zalloc((size_t)s->nn * 8);
  s->lflag = zalloc(s->nn); s->dmask = zalloc(s->nn);
  s->crack_of = (int *)malloc((size_t)s->ne * sizeof(int));
  for (int e = 0; e < s->ne; ++e) s->crack_of[e] = -1;
  s->cr = (orc_crack *)zalloc((size_t)crack_cap * sizeof(orc_crack));
  s->ph = (orc_phantom *)zalloc((size_t)phantom_cap * sizeof(orc_phantom));
  s->gc = (float *)zalloc((size_t)s->ne * sizeof(float));
  s->eps_own = zalloc((size_t)s->ne * 12 * 8);
  s->eps = zalloc((size_t)s->ne * 12 * 8);
  s->sig = zalloc((size_t)s->ne * 12 * 8);
  s->fe = zalloc((size_t)s->ne * 8 * 8);
  s->peps = zalloc((size_t)crack_cap * 24 * 8);
  s->psig = zalloc((size_t)crack_cap * 24 * 8);
  s->pf = zalloc((size_t)crack_cap * 16 * 8);
  s->reccap = 64;
  s->erec = zalloc((size_t)s->reccap * 7 * 8);
  s->gamma = 1.0;
  return s;
}

void orc_destroy(orc_sim *s) {
  if (!s) return;
  free(s->active); free(s->ux); free(s->uy); free(s->vx); free(s->vy);
  free(s->m); free(s->minv); free(s->Wn); free(s->Wd); free(s->fx); free(s->fy);
  free(s->Fx); free(s->Fy); free(s->Vx); free(s->Vy); free(s->lflag);
  free(s->dmask); free(s->crack_of); free(s->cr); free(s->ph); free(s->gc);
  free(s->eps_own); free(s->eps); free(s->sig); free(s->fe); free(s->peps);
  free(s->psig); free(s->pf); free(s->erec);
  free(s);
}

/* ----------------------------------------------------------------- masses */

/* Row-sum lumped mass: every piece (an intact element is one piece with
 * area A) gives rho*A_p/4 to each of its four nodes.  Summed in increasing
 * element id, then piece order. */
static double piece_mass(const orc_sim *s, double Ap) { return s->rho * Ap * 0.25; }

static double mass_real(const orc_sim *s, int N) {
  int r = s->nx + 1, i = N % r, j = N / r;
  static const int di[4] = {-1, 0, -1, 0}, dj[4] = {-1, -1, 0, 0}, la[4] = {2, 3, 1, 0};
  double acc = 0.0;
  for (int q = 0; q < 4; ++q) {
    int ei = i + di[q], ej = j + dj[q];
    if (ei < 0 || ej < 0 || ei >= s->nx || ej >= s->ny) continue;
    int e = ej * s->nx + ei;
    int st = elem_status(s, e);
    if (st == ST_INTACT) acc = acc + piece_mass(s, s->A);
    else if (st == ST_CRACKED) {
      const orc_crack *c = &s->cr[s->crack_of[e]];
      acc = acc + piece_mass(s, c->Ap[c->side[la[q]]]);
    }
  }
  return acc;
}

static double mass_phantom(const orc_sim *s, int P) {
  const orc_phantom *p = &s->ph[P - s->nn];
  double acc = 0.0;
  for (int u = 0; u < p->nuser; ++u) {
    const orc_crack *c = &s->cr[s->crack_of[p->ue[u]]];
    acc = acc + piece_mass(s, c->Ap[p->up[u]]);
  }
  return acc;
}

static void set_mass(orc_sim *s, int N, double m) {
  s->m[N] = m;
  s->minv[N] = m > 0.0 ? 1.0 / m : 0.0;
}

static void recompute_all_masses(orc_sim *s) {
  for (int N = 0; N < s->nn; ++N) set_mass(s, N, mass_real(s, N));
  for (int P = 0; P < s->nph; ++P) set_mass(s, s->nn + P, mass_phantom(s, s->nn + P));
}

/* --------------------------------------------------------------- material */

int orc_set_material(orc_sim *s, double E, double nu, double rho,
                     const float *gc, double gc_uniform, int plane_strain,
                     double gamma, int gamma_mode, int scope) {
  if (!(E > 0) || !(nu > -1.0 && nu < 0.5) || !(rho > 0))
    return fail(s, ORC_ERR_ARG, "bad material");
  if (scope < 0 || scope > 2 || gamma_mode < 0 || gamma_mode > 1)
    return fail(s, ORC_ERR_ARG, "bad scope/gamma mode");
  s->E = E; s->nu = nu; s->rho = rho; s->plane_strain = plane_strain != 0;
  s->gamma = gamma; s->gamma_mode = gamma_mode; s->scope = scope;
  if (s->plane_strain) {
    double c = E / ((1.0 + nu) * (1.0 - 2.0 * nu));
    s->D11 = c * (1.0 - nu);
    s->D12 = c * nu;
    s->D33 = c * (1.0 - 2.0 * nu) * 0.5;
  } else {
    double c = E / (1.0 - nu * nu);
    s->D11 = c;
    s->D12 = c * nu;
    s->D33 = c * (1.0 - nu) * 0.5;
  }
  for (int e = 0; e < s->ne; ++e) s->gc[e] = gc ? gc[e] : (float)gc_uniform;
  s->mat_set = 1;
  recompute_all_masses(s);
  if (!s->dt_set) orc_set_dt(s, 0.5, 0.0);
  return ORC_OK;
}

/* Dilatational wave speed of the plane problem and the explicit step
 * dt = dt_factor * h_min / c_d. */
int orc_set_dt(orc_sim *s, double dt_factor, double dt_explicit) {
  if (!s->mat_set && !(dt_explicit > 0)) return fail(s, ORC_ERR_STATE, "material first");
  if (dt_explicit > 0) {
    s->dt = dt_explicit;
  } else {
    double E = s->E, nu = s->nu, rho = s->rho, cd;
    if (s->plane_strain) cd = sqrt((E * (1.0 - nu)) / (rho * ((1.0 + nu) * (1.0 - 2.0 * nu))));
    else cd = sqrt(E / (rho * (1.0 - nu * nu)));
    double h = s->hx < s->hy ? s->hx : s->hy;
    s->dt = dt_factor * h / cd;
  }
  s->dt_set = 1;
  return ORC_OK;
}

double orc_dt(const orc_sim *s) { return s->dt; }

int orc_set_energy_every(orc_sim *s, int K) {
  s->energy_every = K > 0 ? K : 0;
  return ORC_OK;
}

/* ---------------------------------------------------------------- loads */

/* Outward unit normal of edge g seen from its single active neighbour. */
static int edge_outward(const orc_sim *s, int g, double *nx, double *ny) {
  int lo, klo, hi, khi;
  edge_sides(s, g, &lo, &klo, &hi, &khi);
  int alo = lo >= 0 && s->active[lo], ahi = hi >= 0 && s->active[hi];
  if (alo == ahi) return -1;
  int horiz = g < s->nh;
  double sgn = alo ? 1.0 : -1.0; /* material below/left: normal points +y/+x */
  *nx = horiz ? 0.0 : sgn;
  *ny = horiz ? sgn : 0.0;
  return 0;
}

static void edge_nodes(const orc_sim *s, int g, int *n1, int *n2) {
  int r = s->nx + 1;
  if (g < s->nh) {
    int j = g / s->nx, i = g % s->nx;
    *n1 = j * r + i; *n2 = j * r + i + 1;
  } else {
    int gg = g - s->nh, j = gg / r, i = gg % r;
    *n1 = j * r + i; *n2 = (j + 1) * r + i;
  }
}

/* Neumann loads become equivalent nodal forces: each node of a loaded edge
 * of length L receives L/2 times the traction (Sec. 4.3, last paragraph).
 * The time law multiplies them (Eqs. 7-9 shapes). */
int orc_add_bc(orc_sim *s, int kind, int n, const int *items, int comp_mask,
               int law, double a0, double t0, double tau) {
  if (n < 0 || (n > 0 && !items)) return fail(s, ORC_ERR_ARG, "bad items");
  if (law < 0 || law > 2) return fail(s, ORC_ERR_ARG, "bad law");
  if (law != ORC_LAW_CONST && !(t0 > 0)) return fail(s, ORC_ERR_ARG, "t0 must be > 0");
  if (law == ORC_LAW_RAMP_EXP && !(tau > 0)) return fail(s, ORC_ERR_ARG, "tau must be > 0");
  if (kind == ORC_TRACTION || kind == ORC_PRESSURE) {
    if (s->neu_set && (s->neu_law != law || s->neu_t0 != t0 || s->neu_tau != tau))
      return fail(s, ORC_ERR_ARG, "all Neumann loads share one time law");
    /* validate first */
    for (int q = 0; q < n; ++q) {
      double ox, oy;
      if (items[q] < 0 || items[q] >= s->ned || edge_outward(s, items[q], &ox, &oy))
        return fail(s, ORC_ERR_ARG, "edge %d is not a boundary edge", items[q]);
    }
    int *sorted = (int *)malloc((size_t)(n ? n : 1) * sizeof(int));
    memcpy(sorted, items, (size_t)n * sizeof(int));
    /* insertion sort: loads are added in increasing edge id */
    for (int a = 1; a < n; ++a) {
      int v = sorted[a], b = a - 1;
      while (b >= 0 && sorted[b] > v) { sorted[b + 1] = sorted[b]; --b; }
      sorted[b + 1] = v;
    }
    for (int q = 0; q < n; ++q) {
      int g = sorted[q], n1, n2;
      double ox, oy, tx, ty;
      edge_outward(s, g, &ox, &oy);
      double L = g < s->nh ? s->hx : s->hy;
      if (kind == ORC_TRACTION) {
        tx = (comp_mask & 1) ? a0 : 0.0;
        ty = (comp_mask & 2) ? a0 : 0.0;
      } else { /* pressure pushes into the material */
        tx = -a0 * ox;
        ty = -a0 * oy;
      }
      double half = 0.5 * L;
      edge_nodes(s, g, &n1, &n2);
      s->Fx[n1] = s->Fx[n1] + half * tx; s->Fy[n1] = s->Fy[n1] + half * ty;
      s->Fx[n2] = s->Fx[n2] + half * tx; s->Fy[n2] = s->Fy[n2] + half * ty;
      s->lflag[n1] = 1; s->lflag[n2] = 1;
    }
    free(sorted);
    s->neu_set = 1; s->neu_law = law; s->neu_t0 = t0; s->neu_tau = tau;
    return ORC_OK;
  }
  if (kind == ORC_VELOCITY) {
    if (s->dir_set && (s->dir_law != law || s->dir_t0 != t0 || s->dir_tau != tau))
      return fail(s, ORC_ERR_ARG, "all Dirichlet loads share one time law");
    if ((comp_mask & 3) == 0) return fail(s, ORC_ERR_ARG, "empty component mask");
    for (int q = 0; q < n; ++q)
      if (items[q] < 0 || items[q] >= s->nn) return fail(s, ORC_ERR_ARG, "bad node %d", items[q]);
    for (int q = 0; q < n; ++q) {
      int N = items[q];
      if (comp_mask & 1) { s->dmask[N] |= 1; s->Vx[N] = a0; }
      if (comp_mask & 2) { s->dmask[N] |= 2; s->Vy[N] = a0; }
    }
    s->dir_set = 1; s->dir_law = law; s->dir_t0 = t0; s->dir_tau = tau;
    return ORC_OK;
  }
  return fail(s, ORC_ERR_ARG, "bad kind");
}

int orc_set_state(orc_sim *s, const double *ux, const double *uy,
                  const double *vx, const double *vy) {
  if (s->step != 0) return fail(s, ORC_ERR_STATE, "state can only be set before the first step");
  for (int N = 0; N < s->nn + s->nph; ++N) {
    if (ux) s->ux[N] = ux[N];
    if (uy) s->uy[N] = uy[N];
    if (vx) s->vx[N] = vx[N];
    if (vy) s->vy[N] = vy[N];
  }
  return ORC_OK;
}

/* ------------------------------------------------------- strain and force */

/* eps = B(g_k) u, Eq. 4 evaluated at edge point k: (exx, eyy, gamma_xy). */
static void strain_at(const orc_sim *s, int k, const double ux[4],
                      const double uy[4], double eps[3]) {
  double exx = 0.0, eyy = 0.0, g1 = 0.0, g2 = 0.0;
  for (int a = 0; a < 4; ++a) exx = exx + dNdx(s, k, a) * ux[a];
  for (int a = 0; a < 4; ++a) eyy = eyy + dNdy(s, k, a) * uy[a];
  for (int a = 0; a < 4; ++a) g1 = g1 + dNdy(s, k, a) * ux[a];
  for (int a = 0; a < 4; ++a) g2 = g2 + dNdx(s, k, a) * uy[a];
  eps[0] = exx;
  eps[1] = eyy;
  eps[2] = g1 + g2;
}

static void stress_of(const orc_sim *s, const double eps[3], double sig[3]) {
  sig[0] = s->D11 * eps[0] + s->D12 * eps[1];
  sig[1] = s->D12 * eps[0] + s->D11 * eps[1];
  sig[2] = s->D33 * eps[2];
}

/* f_a = sum_k B_a(g_k)^T sigma_k * A_p/4  (Eq. 6 with w_j * sum A / 4 = A_j/4). */
static void piece_force(const orc_sim *s, const double *sig /* [4][3] */,
                        double Ap, double f[8]) {
  double q = Ap * 0.25;
  for (int a = 0; a < 4; ++a) {
    double sx = 0.0, sy = 0.0;
    for (int k = 0; k < 4; ++k) {
      const double *sg = sig + 3 * k;
      sx = sx + (dNdx(s, k, a) * sg[0] + dNdy(s, k, a) * sg[2]);
      sy = sy + (dNdy(s, k, a) * sg[1] + dNdx(s, k, a) * sg[2]);
    }
    f[2 * a] = sx * q;
    f[2 * a + 1] = sy * q;
  }
}

static void compute_forces(orc_sim *s) {
  int n4[4];
  double ux[4], uy[4];
  /* 1. each intact element's own strain at its four edge points */
  for (int e = 0; e < s->ne; ++e) {
    if (elem_status(s, e) != ST_INTACT) continue;
    elem_nodes(s, e, n4);
    for (int a = 0; a < 4; ++a) { ux[a] = s->ux[n4[a]]; uy[a] = s->uy[n4[a]]; }
    for (int k = 0; k < 4; ++k) strain_at(s, k, ux, uy, s->eps_own + (size_t)e * 12 + 3 * k);
  }
  /* 2. edge strain: area-weighted average over the two intact neighbours
   *    (Eqs. 1-2); own strain on a boundary edge or beside a cracked
   *    element (smoothing off there). */
  for (int e = 0; e < s->ne; ++e) {
    if (elem_status(s, e) != ST_INTACT) continue;
    for (int k = 0; k < 4; ++k) {
      double *ep = s->eps + (size_t)e * 12 + 3 * k;
      const double *own = s->eps_own + (size_t)e * 12 + 3 * k;
      int f = elem_neighbor(s, e, k);
      if (elem_status(s, f) == ST_INTACT) {
        int kf = (k + 2) % 4;
        int e1 = e < f ? e : f, k1 = e < f ? k : kf;
        int e2 = e < f ? f : e, k2 = e < f ? kf : k;
        double A1 = s->A, A2 = s->A;
        double w1 = A1 / (A1 + A2), w2 = A2 / (A1 + A2);
        const double *p1 = s->eps_own + (size_t)e1 * 12 + 3 * k1;
        const double *p2 = s->eps_own + (size_t)e2 * 12 + 3 * k2;
        for (int c = 0; c < 3; ++c) ep[c] = w1 * p1[c] + w2 * p2[c];
      } else {
        for (int c = 0; c < 3; ++c) ep[c] = own[c];
      }
      stress_of(s, ep, s->sig + (size_t)e * 12 + 3 * k);
    }
    piece_force(s, s->sig + (size_t)e * 12, s->A, s->fe + (size_t)e * 8);
  }
  /* 3. split pieces: own strain, own stress, force scaled by the piece area */
  for (int c = 0; c < s->ncr; ++c) {
    const orc_crack *cr = &s->cr[c];
    for (int p = 0; p < 2; ++p) {
      for (int a = 0; a < 4; ++a) { ux[a] = s->ux[cr->node[p][a]]; uy[a] = s->uy[cr->node[p][a]]; }
      double *pe = s->peps + (size_t)c * 24 + p * 12;
      double *ps = s->psig + (size_t)c * 24 + p * 12;
      for (int k = 0; k < 4; ++k) {
        strain_at(s, k, ux, uy, pe + 3 * k);
        stress_of(s, pe + 3 * k, ps + 3 * k);
      }
      piece_force(s, ps, cr->Ap[p], s->pf + (size_t)c * 16 + p * 8);
    }
  }
  /* 4. nodal internal force: sum over (element, piece, local node) slots in
   *    increasing element id */
  static const int di[4] = {-1, 0, -1, 0}, dj[4] = {-1, -1, 0, 0}, la[4] = {2, 3, 1, 0};
  int r = s->nx + 1;
  for (int N = 0; N < s->nn; ++N) {
    int i = N % r, j = N / r;
    double ax = 0.0, ay = 0.0;
    for (int q = 0; q < 4; ++q) {
      int ei = i + di[q], ej = j + dj[q];
      if (ei < 0 || ej < 0 || ei >= s->nx || ej >= s->ny) continue;
      int e = ej * s->nx + ei, a = la[q], st = elem_status(s, e);
      if (st == ST_INTACT) {
        ax = ax + s->fe[(size_t)e * 8 + 2 * a];
        ay = ay + s->fe[(size_t)e * 8 + 2 * a + 1];
      } else if (st == ST_CRACKED) {
        int c = s->crack_of[e], p = s->cr[c].side[a];
        ax = ax + s->pf[(size_t)c * 16 + p * 8 + 2 * a];
        ay = ay + s->pf[(size_t)c * 16 + p * 8 + 2 * a + 1];
      }
    }
    s->fx[N] = ax;
    s->fy[N] = ay;
  }
  for (int P = 0; P < s->nph; ++P) {
    const orc_phantom *ph = &s->ph[P];
    double ax = 0.0, ay = 0.0;
    for (int u = 0; u < ph->nuser; ++u) {
      int c = s->crack_of[ph->ue[u]];
      ax = ax + s->pf[(size_t)c * 16 + ph->up[u] * 8 + 2 * ph->ua[u]];
      ay = ay + s->pf[(size_t)c * 16 + ph->up[u] * 8 + 2 * ph->ua[u] + 1];
    }
    s->fx[s->nn + P] = ax;
    s->fy[s->nn + P] = ay;
  }
}

/* Strain energy: each element (or piece) owns A_p/4 of each of its edge
 * points; SE = sum 1/2 (A_p/4) eps . sigma, in element order. */
static double strain_energy(const orc_sim *s) {
  double se = 0.0;
  for (int e = 0; e < s->ne; ++e) {
    int st = elem_status(s, e);
    if (st == ST_INTACT) {
      double q = s->A * 0.25, acc = 0.0;
      for (int k = 0; k < 4; ++k) {
        const double *ep = s->eps + (size_t)e * 12 + 3 * k, *sg = s->sig + (size_t)e * 12 + 3 * k;
        double d = ep[0] * sg[0] + ep[1] * sg[1] + ep[2] * sg[2];
        acc = acc + 0.5 * (q * d);
      }
      se = se + acc;
    } else if (st == ST_CRACKED) {
      int c = s->crack_of[e];
      double acc = 0.0;
      for (int p = 0; p < 2; ++p) {
        double q = s->cr[c].Ap[p] * 0.25;
        for (int k = 0; k < 4; ++k) {
          const double *ep = s->peps + (size_t)c * 24 + p * 12 + 3 * k;
          const double *sg = s->psig + (size_t)c * 24 + p * 12 + 3 * k;
          double d = ep[0] * sg[0] + ep[1] * sg[1] + ep[2] * sg[2];
          acc = acc + 0.5 * (q * d);
        }
      }
      se = se + acc;
    }
  }
  return se;
}

/* ------------------------------------------------------- crack geometry */

/* Midpoint of local edge k relative to the element's lower-left corner. */
static void mid_phys(const orc_sim *s, int k, double *x, double *y) {
  *x = (XI_G[k] + 1.0) * (0.5 * s->hx);
  *y = (ETA_G[k] + 1.0) * (0.5 * s->hy);
}

/* Reference vector X_N2 - X_N1 of local edge k, N1 = local node k,
 * N2 = local node (k+1)%4. */
static void edge_vec(const orc_sim *s, int k, double *dx, double *dy) {
  *dx = (XI_N[(k + 1) % 4] - XI_N[k]) * (0.5 * s->hx);
  *dy = (ETA_N[(k + 1) % 4] - ETA_N[k]) * (0.5 * s->hy);
}

/* Energy release rate of the candidate paths from the surface point on local
 * edge k0 of intact element e to its other three edge points (Sec. 2.2).
 * G[k0] is set to -1. */
static void eval_G(const orc_sim *s, int e, int k0, double G[4]) {
  int n4[4];
  elem_nodes(s, e, n4);
  int N1 = n4[k0], N2 = n4[(k0 + 1) % 4];
  double DX, DY;
  edge_vec(s, k0, &DX, &DY);
  double dux = s->ux[N2] - s->ux[N1];
  double duy = s->uy[N2] - s->uy[N1];
  double dx = DX + dux, dy = DY + duy;
  double cur2 = dx * dx + dy * dy;
  double ref2 = DX * DX + DY * DY;
  /* Heaviside of (|x_N2-x_N1|/|X_N2-X_N1| - 1): 1 only for a stretched edge */
  double H = cur2 > ref2 ? 1.0 : 0.0;
  double ddx = dux * H, ddy = duy * H;
  double x0, y0;
  mid_phys(s, k0, &x0, &y0);
  for (int k = 0; k < 4; ++k) {
    if (k == k0) { G[k] = -1.0; continue; }
    double xk, yk;
    mid_phys(s, k, &xk, &yk);
    double sx = xk - x0, sy = yk - y0;
    /* unit normal of the segment G0->Gk, oriented along X_N2 - X_N1 */
    double rx = -sy, ry = sx;
    if (rx * DX + ry * DY < 0.0) { rx = -rx; ry = -ry; }
    double len = sqrt(sx * sx + sy * sy);
    double nx = rx / len, ny = ry / len;
    const double *sg = s->sig + (size_t)e * 12 + 3 * k;
    double tx = sg[0] * nx + sg[2] * ny;
    double ty = sg[2] * nx + sg[1] * ny;
    G[k] = 0.5 * (ddx * tx + ddy * ty);
  }
}

/* Q4 cracking conditions (Sec. 2.2): none, one or several candidates above
 * G_c; with several, the largest p must satisfy the split-ratio test
 * against every other candidate q above G_c. Returns the chosen edge or -1. */
static int q4_rule(const orc_sim *s, int e, int k0, const double G[4]) {
  double gc = (double)s->gc[e];
  int best = -1, ncand = 0;
  for (int k = 0; k < 4; ++k) {
    if (k == k0 || !(G[k] > gc)) continue;
    ++ncand;
    if (best < 0 || G[k] > G[best]) best = k;
  }
  if (ncand == 0) return -1;
  for (int q = 0; q < 4; ++q) {
    if (q == k0 || q == best || !(G[q] > gc)) continue;
    int ok = s->gamma_mode == ORC_GAMMA_LITERAL ? (G[best] > s->gamma * (G[best] - G[q]))
                                                : (G[best] > s->gamma * G[q]);
    if (!ok) return -1;
  }
  return best;
}

/* Surface set: every edge with exactly one intact neighbour (the element
 * "ahead" of the edge point).  A tip is a surface edge that is a cut edge
 * of the cracked element on its other side. */
static int surface_info(const orc_sim *s, int g, int *ahead, int *k0, int *is_tip) {
  int lo, klo, hi, khi;
  edge_sides(s, g, &lo, &klo, &hi, &khi);
  int slo = elem_status(s, lo), shi = elem_status(s, hi);
  if ((slo == ST_INTACT) == (shi == ST_INTACT)) return 0;
  int other, kother;
  if (slo == ST_INTACT) { *ahead = lo; *k0 = klo; other = hi; kother = khi; }
  else { *ahead = hi; *k0 = khi; other = lo; kother = klo; }
  *is_tip = 0;
  if (elem_status(s, other) == ST_CRACKED) {
    const orc_crack *c = &s->cr[s->crack_of[other]];
    *is_tip = (c->ka == kother || c->kb == kother);
  }
  return 1;
}

/* ----------------------------------------------------------------- split */

static int local_index(const int n4[4], int N) {
  for (int a = 0; a < 4; ++a)
    if (n4[a] == N) return a;
  return -1;
}

static int add_user(orc_sim *s, int P, int e, int p, int a) {
  orc_phantom *ph = &s->ph[P - s->nn];
  if (ph->nuser >= 4) return fail(s, ORC_ERR_CAPACITY, "phantom user overflow");
  int q = ph->nuser;
  while (q > 0 && ph->ue[q - 1] > e) {
    ph->ue[q] = ph->ue[q - 1]; ph->up[q] = ph->up[q - 1]; ph->ua[q] = ph->ua[q - 1];
    --q;
  }
  ph->ue[q] = e; ph->up[q] = p; ph->ua[q] = a;
  ph->nuser++;
  return ORC_OK;
}

/* Split intact element e along the segment from the midpoint of local edge
 * ka to that of kb (crack patterns I and II, Fig. 2-3) into two phantom-node
 * pieces.  A phantom is shared with the cracked neighbour across a cut edge
 * that contains its real node. */
static int split_element(orc_sim *s, int e, int ka, int kb, int step, int precrack) {
  if (elem_status(s, e) != ST_INTACT) return fail(s, ORC_ERR_STATE, "element %d not intact", e);
  if (ka == kb || ka < 0 || kb < 0 || ka > 3 || kb > 3) return fail(s, ORC_ERR_ARG, "bad cut edges");
  if (s->ncr >= s->crcap) return fail(s, ORC_ERR_CAPACITY, "crack table full");
  int n4[4];
  elem_nodes(s, e, n4);
  int c = s->ncr;
  orc_crack *cr = &s->cr[c];
  memset(cr, 0, sizeof *cr);
  cr->elem = e; cr->ka = ka; cr->kb = kb; cr->step = precrack ? -1 : step;
  double pax = XI_G[ka], pay = ETA_G[ka], pbx = XI_G[kb], pby = ETA_G[kb];
  for (int a = 0; a < 4; ++a) {
    double cross = (pbx - pax) * (ETA_N[a] - pay) - (pby - pay) * (XI_N[a] - pax);
    cr->side[a] = cross > 0.0 ? 0 : 1;
  }
  /* area fractions by the shoelace formula in natural coordinates
   * (area of the reference square is 4) */
  for (int p = 0; p < 2; ++p) {
    double px[6], py[6];
    int nv = 0;
    for (int w = 0; w < 8; ++w) {
      if (w % 2 == 0) {
        int a = w / 2;
        if (cr->side[a] == p) { px[nv] = XI_N[a]; py[nv] = ETA_N[a]; ++nv; }
      } else {
        int k = w / 2;
        if (k == ka || k == kb) { px[nv] = XI_G[k]; py[nv] = ETA_G[k]; ++nv; }
      }
    }
    double twice = 0.0;
    for (int v = 0; v < nv; ++v) {
      int w = (v + 1) % nv;
      twice = twice + (px[v] * py[w] - px[w] * py[v]);
    }
    cr->alpha[p] = fabs(twice) * 0.5 / 4.0;
    cr->Ap[p] = cr->alpha[p] * s->A;
  }
  for (int a = 0; a < 4; ++a) cr->node[cr->side[a]][a] = n4[a];
  /* phantom nodes in increasing local node order */
  int reused[4] = {-1, -1, -1, -1};
  double mold[4] = {0, 0, 0, 0};
  for (int a = 0; a < 4; ++a) {
    int p = 1 - cr->side[a];
    int P = -1;
    int kk[2] = {(a + 3) % 4, a};
    if (kk[0] > kk[1]) { int t = kk[0]; kk[0] = kk[1]; kk[1] = t; }
    for (int q = 0; q < 2 && P < 0; ++q) {
      int k = kk[q];
      if (k != ka && k != kb) continue;
      int f = elem_neighbor(s, e, k);
      if (elem_status(s, f) != ST_CRACKED) continue;
      const orc_crack *cf = &s->cr[s->crack_of[f]];
      int kf = (k + 2) % 4;
      if (cf->ka != kf && cf->kb != kf) continue;
      int nf[4];
      elem_nodes(s, f, nf);
      int af = local_index(nf, n4[a]);
      P = cf->node[1 - cf->side[af]][af];
    }
    if (P < 0) {
      if (s->nph >= s->phcap) return fail(s, ORC_ERR_CAPACITY, "phantom pool full");
      P = s->nn + s->nph;
      orc_phantom *ph = &s->ph[s->nph++];
      memset(ph, 0, sizeof *ph);
      ph->owner = n4[a]; ph->creator_e = e; ph->creator_a = a;
      s->ux[P] = s->ux[n4[a]]; s->uy[P] = s->uy[n4[a]];
      s->vx[P] = s->vx[n4[a]]; s->vy[P] = s->vy[n4[a]];
      s->Wn[P] = 0.0; s->Wd[P] = 0.0;
    } else {
      reused[a] = P;
      mold[a] = s->m[P];
    }
    cr->node[p][a] = P;
  }
  s->crack_of[e] = c;
  s->ncr++;
  for (int a = 0; a < 4; ++a) {
    int rc = add_user(s, cr->node[1 - cr->side[a]][a], e, 1 - cr->side[a], a);
    if (rc) return rc;
  }
  /* masses of the real nodes and phantoms touched by the split */
  for (int a = 0; a < 4; ++a) set_mass(s, n4[a], mass_real(s, n4[a]));
  for (int a = 0; a < 4; ++a) {
    int P = cr->node[1 - cr->side[a]][a];
    double mnew = mass_phantom(s, P);
    if (reused[a] >= 0) {
      /* momentum-conserving merge of the mass moved from the real node */
      double dm = piece_mass(s, cr->Ap[1 - cr->side[a]]);
      int N = n4[a];
      s->vx[P] = (mold[a] * s->vx[P] + dm * s->vx[N]) / mnew;
      s->vy[P] = (mold[a] * s->vy[P] + dm * s->vy[N]) / mnew;
    }
    set_mass(s, P, mnew);
  }
  if (!precrack) {
    double xa, ya, xb, yb;
    mid_phys(s, ka, &xa, &ya);
    mid_phys(s, kb, &xb, &yb);
    double sx = xb - xa, sy = yb - ya;
    double L = sqrt(sx * sx + sy * sy);
    cr->ud = (double)s->gc[e] * L;
  }
  return ORC_OK;
}

int orc_precrack(orc_sim *s, int n, const int *t) {
  if (!s->mat_set) return fail(s, ORC_ERR_STATE, "material first");
  for (int q = 0; q < n; ++q) {
    int e = t[3 * q];
    if (e < 0 || e >= s->ne || !s->active[e]) return fail(s, ORC_ERR_ARG, "bad precrack element");
    int rc = split_element(s, e, t[3 * q + 1], t[3 * q + 2], 0, 1);
    if (rc) return rc;
  }
  return ORC_OK;
}

/* ------------------------------------------------------------ selection */

typedef struct { int edge, elem, k; double G; } proposal;

static int key_greater(const proposal *a, const proposal *b) {
  return a->G > b->G || (a->G == b->G && a->edge < b->edge);
}

static int near_elems(const orc_sim *s, int e, int f) {
  int di = e % s->nx - f % s->nx, dj = e / s->nx - f / s->nx;
  return di >= -1 && di <= 1 && dj >= -1 && dj <= 1;
}

/* Multiple Crack-tips Tracking selection (Sec. 3): the largest G among the
 * candidates wins.  Scope NBHD: a proposal wins if its key (G, -edge) is the
 * strict maximum among proposals whose ahead elements share a node with its
 * own; GLOBAL: one winner in the mesh; TIPS: only crack fronts propose. */
static int select_and_split(orc_sim *s, proposal *pr, int np, int step) {
  int *win = (int *)zalloc((size_t)(np ? np : 1) * sizeof(int));
  if (s->scope == ORC_SCOPE_GLOBAL) {
    int b = -1;
    for (int p = 0; p < np; ++p)
      if (b < 0 || key_greater(&pr[p], &pr[b])) b = p;
    if (b >= 0) win[b] = 1;
  } else {
    for (int p = 0; p < np; ++p) {
      int ok = 1;
      for (int q = 0; q < np && ok; ++q)
        if (q != p && near_elems(s, pr[p].elem, pr[q].elem) && !key_greater(&pr[p], &pr[q])) ok = 0;
      win[p] = ok;
    }
  }
  /* apply in increasing element id */
  int rc = ORC_OK;
  for (;;) {
    int b = -1;
    for (int p = 0; p < np; ++p)
      if (win[p] && (b < 0 || pr[p].elem < pr[b].elem)) b = p;
    if (b < 0) break;
    win[b] = 0;
    rc = split_element(s, pr[b].elem, pr[b].edge == elem_edge_id(s, pr[b].elem, 0) ? 0 :
                                      pr[b].edge == elem_edge_id(s, pr[b].elem, 1) ? 1 :
                                      pr[b].edge == elem_edge_id(s, pr[b].elem, 2) ? 2 : 3,
                       pr[b].k, step, 0);
    if (rc) break;
  }
  free(win);
  return rc;
}

static int gather_proposals(orc_sim *s, proposal **out) {
  int cap = 64, np = 0;
  proposal *pr = (proposal *)malloc((size_t)cap * sizeof *pr);
  for (int g = 0; g < s->ned; ++g) {
    int e, k0, tip;
    if (!surface_info(s, g, &e, &k0, &tip)) continue;
    if (s->scope == ORC_SCOPE_TIPS && !tip) continue;
    double G[4];
    eval_G(s, e, k0, G);
    int k = q4_rule(s, e, k0, G);
    if (k < 0) continue;
    if (np == cap) { cap *= 2; pr = (proposal *)realloc(pr, (size_t)cap * sizeof *pr); }
    pr[np].edge = g; pr[np].elem = e; pr[np].k = k; pr[np].G = G[k];
    ++np;
  }
  *out = pr;
  return np;
}

/* ------------------------------------------------------------------ step */

static double ud_total(const orc_sim *s) {
  double acc = 0.0;
  for (int e = 0; e < s->ne; ++e)
    if (s->active[e] && s->crack_of[e] >= 0) acc = acc + s->cr[s->crack_of[e]].ud;
  return acc;
}

static int do_step(orc_sim *s) {
  int n = s->step;
  int nall = s->nn + s->nph;
  double dt = s->dt;
  double t = (double)n * dt;
  compute_forces(s);
  proposal *pr = NULL;
  int np = gather_proposals(s, &pr);
  int energy = s->energy_every > 0 && n % s->energy_every == 0;
  double Wn_tot = 0.0, Wd_tot = 0.0, KE = 0.0, SE = 0.0;
  if (energy) {
    for (int N = 0; N < nall; ++N) { Wn_tot = Wn_tot + s->Wn[N]; Wd_tot = Wd_tot + s->Wd[N]; }
    SE = strain_energy(s);
  }
  double lamN = s->neu_set ? law_eval(s->neu_law, t, s->neu_t0, s->neu_tau) : 0.0;
  double lamD = s->dir_set ? law_eval(s->dir_law, ((double)n + 0.5) * dt, s->dir_t0, s->dir_tau) : 0.0;
  double dtv = n == 0 ? 0.5 * dt : dt;
  /* central-difference update with half-step velocities */
  for (int N = 0; N < nall; ++N) {
    int real = N < s->nn;
    int loaded = real && s->lflag[N];
    int dm = real ? s->dmask[N] : 0;
    double fex = loaded ? lamN * s->Fx[N] : 0.0;
    double fey = loaded ? lamN * s->Fy[N] : 0.0;
    double ax = (fex - s->fx[N]) * s->minv[N];
    double ay = (fey - s->fy[N]) * s->minv[N];
    double vxo = s->vx[N], vyo = s->vy[N];
    double vxn = vxo + dtv * ax;
    double vyn = vyo + dtv * ay;
    if (dm & 1) vxn = lamD * s->Vx[N];
    if (dm & 2) vyn = lamD * s->Vy[N];
    double vbx = n == 0 ? vxo : 0.5 * (vxo + vxn);
    double vby = n == 0 ? vyo : 0.5 * (vyo + vyn);
    if (loaded) s->Wn[N] = s->Wn[N] + dt * (fex * vbx + fey * vby);
    if (dm) {
      double Rx = s->m[N] * ((vxn - vxo) / dtv) - (fex - s->fx[N]);
      double Ry = s->m[N] * ((vyn - vyo) / dtv) - (fey - s->fy[N]);
      double w = 0.0;
      if (dm & 1) w = w + Rx * vbx;
      if (dm & 2) w = w + Ry * vby;
      s->Wd[N] = s->Wd[N] + dt * w;
    }
    if (energy) KE = KE + 0.5 * (s->m[N] * (vbx * vbx + vby * vby));
    s->vx[N] = vxn;
    s->vy[N] = vyn;
    s->ux[N] = s->ux[N] + dt * vxn;
    s->uy[N] = s->uy[N] + dt * vyn;
  }
  if (energy) {
    if (s->nrec == s->reccap) {
      s->reccap *= 2;
      s->erec = (double *)realloc(s->erec, (size_t)s->reccap * 7 * 8);
    }
    double *r = s->erec + (size_t)s->nrec * 7;
    r[0] = (double)n; r[1] = t; r[2] = KE; r[3] = SE; r[4] = Wn_tot; r[5] = Wd_tot; r[6] = ud_total(s);
    s->nrec++;
  }
  int rc = select_and_split(s, pr, np, n);
  free(pr);
  s->step = n + 1;
  return rc;
}

int orc_step(orc_sim *s, int nsteps) {
  if (!s->mat_set) return fail(s, ORC_ERR_STATE, "material first");
  for (int q = 0; q < nsteps; ++q) {
    int rc = do_step(s);
    if (rc) return rc;
  }
  return ORC_OK;
}

/* --------------------------------------------------------------- getters */

void orc_counts(const orc_sim *s, long out[9]) {
  long nS = 0, nT = 0;
  for (int g = 0; g < s->ned; ++g) {
    int e, k0, tip;
    if (surface_info(s, g, &e, &k0, &tip)) { ++nS; nT += tip; }
  }
  out[0] = s->nn; out[1] = s->ne; out[2] = s->ned; out[3] = s->nph; out[4] = s->ncr;
  out[5] = s->step; out[6] = nS; out[7] = nT; out[8] = s->nrec;
}

int orc_get_nodes(const orc_sim *s, double *ux, double *uy, double *vx, double *vy, double *m) {
  int n = s->nn + s->nph;
  for (int N = 0; N < n; ++N) {
    if (ux) ux[N] = s->ux[N];
    if (uy) uy[N] = s->uy[N];
    if (vx) vx[N] = s->vx[N];
    if (vy) vy[N] = s->vy[N];
    if (m) m[N] = s->m[N];
  }
  return n;
}

int orc_get_phantoms(const orc_sim *s, int *owner, int *ce, int *ca, int *nuser, int *users) {
  for (int P = 0; P < s->nph; ++P) {
    const orc_phantom *ph = &s->ph[P];
    if (owner) owner[P] = ph->owner;
    if (ce) ce[P] = ph->creator_e;
    if (ca) ca[P] = ph->creator_a;
    if (nuser) nuser[P] = ph->nuser;
    if (users)
      for (int u = 0; u < 4; ++u) {
        users[P * 12 + 3 * u] = u < ph->nuser ? ph->ue[u] : -1;
        users[P * 12 + 3 * u + 1] = u < ph->nuser ? ph->up[u] : -1;
        users[P * 12 + 3 * u + 2] = u < ph->nuser ? ph->ua[u] : -1;
      }
  }
  return s->nph;
}

int orc_get_cracks(const orc_sim *s, int *elem, int *ka, int *kb, int *step, double *ud, int *nodes) {
  int q = 0;
  for (int e = 0; e < s->ne; ++e) {
    int c = s->crack_of[e];
    if (c < 0) continue;
    const orc_crack *cr = &s->cr[c];
    if (elem) elem[q] = e;
    if (ka) ka[q] = cr->ka;
    if (kb) kb[q] = cr->kb;
    if (step) step[q] = cr->step;
    if (ud) ud[q] = cr->ud;
    if (nodes)
      for (int p = 0; p < 2; ++p)
        for (int a = 0; a < 4; ++a) nodes[q * 8 + p * 4 + a] = cr->node[p][a];
    ++q;
  }
  return q;
}

int orc_get_surface(const orc_sim *s, int *edge, int *ahead, int *is_tip) {
  int q = 0;
  for (int g = 0; g < s->ned; ++g) {
    int e, k0, tip;
    if (!surface_info(s, g, &e, &k0, &tip)) continue;
    if (edge) edge[q] = g;
    if (ahead) ahead[q] = e;
    if (is_tip) is_tip[q] = tip;
    ++q;
  }
  return q;
}

int orc_get_energy(const orc_sim *s, double *rec) {
  if (rec) memcpy(rec, s->erec, (size_t)s->nrec * 7 * 8);
  return s->nrec;
}

int orc_internal_force(orc_sim *s, double *fx, double *fy) {
  if (!s->mat_set) return fail(s, ORC_ERR_STATE, "material first");
  compute_forces(s);
  int n = s->nn + s->nph;
  memcpy(fx, s->fx, (size_t)n * 8);
  memcpy(fy, s->fy, (size_t)n * 8);
  return n;
}

int orc_strain_energy(orc_sim *s, double *se) {
  if (!s->mat_set) return fail(s, ORC_ERR_STATE, "material first");
  compute_forces(s);
  *se = strain_energy(s);
  return ORC_OK;
}

/* Mean stress of every element: an intact element averages, over its four
 * edge points, the stress its internal force uses there (Eqs. 1-2 edge
 * smoothing applied, Eq. 6); a split element weights its two pieces' mean
 * stresses by the piece areas; an inactive element gets 0.  This is the
 * element stress of the paper's stress contour plots (Sec. 4). */
int orc_element_stress(orc_sim *s, double *sxx, double *syy, double *sxy) {
  if (!s->mat_set) return fail(s, ORC_ERR_STATE, "material first");
  compute_forces(s);
  for (int e = 0; e < s->ne; ++e) {
    double m[3] = {0.0, 0.0, 0.0};
    int st = elem_status(s, e);
    if (st == ST_INTACT) {
      for (int c = 0; c < 3; ++c) {
        const double *sg = s->sig + (size_t)e * 12 + c;
        m[c] = (((sg[0] + sg[3]) + sg[6]) + sg[9]) * 0.25;
      }
    } else if (st == ST_CRACKED) {
      const orc_crack *cr = &s->cr[s->crack_of[e]];
      for (int c = 0; c < 3; ++c) {
        const double *p0 = s->psig + (size_t)s->crack_of[e] * 24 + c;
        const double *p1 = p0 + 12;
        double m0 = (((p0[0] + p0[3]) + p0[6]) + p0[9]) * 0.25;
        double m1 = (((p1[0] + p1[3]) + p1[6]) + p1[9]) * 0.25;
        m[c] = (cr->Ap[0] * m0 + cr->Ap[1] * m1) / (cr->Ap[0] + cr->Ap[1]);
      }
    }
    sxx[e] = m[0];
    syy[e] = m[1];
    sxy[e] = m[2];
  }
  return ORC_OK;
}

int orc_eval_surface(orc_sim *s, int *edge, int *ahead, int *k0out, double *G4, int *prop_k) {
  if (!s->mat_set) return fail(s, ORC_ERR_STATE, "material first");
  compute_forces(s);
  int q = 0;
  for (int g = 0; g < s->ned; ++g) {
    int e, k0, tip;
    if (!surface_info(s, g, &e, &k0, &tip)) continue;
    double G[4];
    eval_G(s, e, k0, G);
    if (edge) edge[q] = g;
    if (ahead) ahead[q] = e;
    if (k0out) k0out[q] = k0;
    if (G4) memcpy(G4 + 4 * q, G, sizeof G);
    if (prop_k) prop_k[q] = q4_rule(s, e, k0, G);
    ++q;
  }
  return q;
}

int orc_apply_proposals(orc_sim *s, int n, const int *edge, const int *elem,
                        const int *k, const double *G) {
  proposal *pr = (proposal *)zalloc((size_t)(n ? n : 1) * sizeof *pr);
  int m = 0;
  for (int q = 0; q < n; ++q) {
    int e, k0, tip;
    if (!surface_info(s, edge[q], &e, &k0, &tip) || e != elem[q] || k[q] == k0 || k[q] < 0 || k[q] > 3) {
      free(pr);
      return fail(s, ORC_ERR_ARG, "proposal %d is not a surface point of its element", q);
    }
    if (s->scope == ORC_SCOPE_TIPS && !tip) continue;
    pr[m].edge = edge[q]; pr[m].elem = elem[q]; pr[m].k = k[q]; pr[m].G = G[q];
    ++m;
  }
  int rc = select_and_split(s, pr, m, s->step);
  free(pr);
  return rc;
}
