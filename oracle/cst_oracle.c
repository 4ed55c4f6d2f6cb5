/*
 * cst_oracle.c -- TEST INFRASTRUCTURE ONLY (see cst_oracle.h).
 *
 * One explicit step of ES-FEM constant-strain triangles, in the paper's
 * order (Sec. 2.1):
 *   1. element strain eps_e = B_e u_e (constant over the triangle);
 *   2. edge strain: on an edge shared by two triangles the area-weighted
 *      average of their strains, w_j = A_j / (A_1 + A_2) (Eqs. 1, 3); on a
 *      boundary edge the one triangle's strain;
 *   3. edge stress sigma_g = D eps_g;
 *   4. internal force: every triangle j of edge g gives its three nodes
 *      B_j^T sigma_g A_j / 3 (Eq. 5: the triangle's third of its area is the
 *      share of the edge's smoothing domain), summed in increasing edge id,
 *      then element id, then local node;
 *   5. central differences with half-step velocities and lumped masses
 *      rho A / 3 per node, the same load laws, prescribed velocities and
 *      energy records as the Q4 oracle.
 * Compiled with -ffp-contract=off: every a*b + c is two roundings.
 */
#include "cst_oracle.h"

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

struct ocst {
  int nn, ne, ned;
  double *X;             /* [2 nn] */
  int *conn;             /* [3 ne] */
  double *A;             /* [ne] areas */
  double *b, *c;         /* [3 ne] dN/dx, dN/dy of the three nodes */
  int *en1, *en2, *ee1, *ee2; /* [ned] edge nodes and elements */
  double E, nu, rho, D11, D12, D33;
  int plane_strain, mat_set, dt_set;
  double dt, hmin;
  double *ux, *uy, *vx, *vy, *m, *minv, *fx, *fy;
  double *eps_e;         /* [3 ne] */
  double *eps_g, *sig_g; /* [3 ned] */
  /* loads */
  double *Fx, *Fy, *Vx, *Vy, *Wn, *Wd;
  unsigned char *lflag, *dmask;
  int neu_set, neu_law, dir_set, dir_law;
  double neu_t0, neu_tau, dir_t0, dir_tau;
  float *gc;             /* [ne] critical energy release rate */
  double gamma;
  int gamma_mode;
  int step, energy_every, nrec, reccap;
  double *erec;
  char err[256];
};

static char g_create_err[256];

const char *ocst_create_error(void) { return g_create_err; }
const char *ocst_error(const ocst *s) { return s->err; }

static int fail(ocst *s, int code, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(s->err, sizeof s->err, fmt, ap);
  va_end(ap);
  return code;
}

static void *zalloc(size_t n) { return calloc(n ? n : 1, 1); }

/* sort keys: edge (min node, max node), then element, then local edge */
typedef struct { int a, b, e, k; } half_edge;

static int cmp_half(const void *p, const void *q) {
  const half_edge *x = (const half_edge *)p, *y = (const half_edge *)q;
  if (x->a != y->a) return x->a < y->a ? -1 : 1;
  if (x->b != y->b) return x->b < y->b ? -1 : 1;
  if (x->e != y->e) return x->e < y->e ? -1 : 1;
  return x->k < y->k ? -1 : (x->k > y->k);
}

void ocst_destroy(ocst *s) {
  if (!s) return;
  void *p[] = {s->gc, s->X, s->conn, s->A, s->b, s->c, s->en1, s->en2, s->ee1, s->ee2, s->ux, s->uy,
               s->vx, s->vy, s->m, s->minv, s->fx, s->fy, s->eps_e, s->eps_g, s->sig_g, s->Fx,
               s->Fy, s->Vx, s->Vy, s->Wn, s->Wd, s->lflag, s->dmask, s->erec};
  for (size_t q = 0; q < sizeof p / sizeof p[0]; ++q) free(p[q]);
  free(s);
}

ocst *ocst_create(int nn, int ne, const double *X, const int *conn) {
  if (nn < 3 || ne < 1 || !X || !conn) {
    snprintf(g_create_err, sizeof g_create_err, "need >= 3 nodes, >= 1 element, X and conn");
    return NULL;
  }
  for (int q = 0; q < 3 * ne; ++q)
    if (conn[q] < 0 || conn[q] >= nn) {
      snprintf(g_create_err, sizeof g_create_err, "node id %d out of range", conn[q]);
      return NULL;
    }
  ocst *s = (ocst *)zalloc(sizeof(ocst));
  s->nn = nn;
  s->ne = ne;
  s->X = (double *)zalloc((size_t)nn * 2 * 8);
  memcpy(s->X, X, (size_t)nn * 2 * 8);
  s->conn = (int *)zalloc((size_t)ne * 3 * 4);
  memcpy(s->conn, conn, (size_t)ne * 3 * 4);
  s->A = (double *)zalloc((size_t)ne * 8);
  s->b = (double *)zalloc((size_t)ne * 3 * 8);
  s->c = (double *)zalloc((size_t)ne * 3 * 8);
  /* geometry: area and shape-function derivatives of each triangle */
  double hmin = INFINITY;
  for (int e = 0; e < ne; ++e) {
    const int *n = conn + 3 * e;
    double x[3], y[3];
    for (int i = 0; i < 3; ++i) { x[i] = X[2 * n[i]]; y[i] = X[2 * n[i] + 1]; }
    double twoA = (x[1] - x[0]) * (y[2] - y[0]) - (x[2] - x[0]) * (y[1] - y[0]);
    if (!(twoA > 0)) {
      snprintf(g_create_err, sizeof g_create_err, "element %d is not counter-clockwise", e);
      ocst_destroy(s);
      return NULL;
    }
    s->A[e] = 0.5 * twoA;
    for (int i = 0; i < 3; ++i) {
      int j = (i + 1) % 3, k = (i + 2) % 3;
      s->b[3 * e + i] = (y[j] - y[k]) / twoA;
      s->c[3 * e + i] = (x[k] - x[j]) / twoA;
    }
    double Lmax = 0.0;
    for (int i = 0; i < 3; ++i) {
      int j = (i + 1) % 3;
      double L = sqrt((x[j] - x[i]) * (x[j] - x[i]) + (y[j] - y[i]) * (y[j] - y[i]));
      if (L > Lmax) Lmax = L;
    }
    double h = twoA / Lmax;
    if (h < hmin) hmin = h;
  }
  s->hmin = hmin;
  /* edges: the distinct node pairs, in increasing (min, max) */
  half_edge *he = (half_edge *)zalloc((size_t)ne * 3 * sizeof(half_edge));
  for (int e = 0; e < ne; ++e)
    for (int k = 0; k < 3; ++k) {
      int a = conn[3 * e + k], b = conn[3 * e + (k + 1) % 3];
      half_edge h = {a < b ? a : b, a < b ? b : a, e, k};
      he[3 * e + k] = h;
    }
  qsort(he, (size_t)ne * 3, sizeof(half_edge), cmp_half);
  s->en1 = (int *)zalloc((size_t)ne * 3 * 4);
  s->en2 = (int *)zalloc((size_t)ne * 3 * 4);
  s->ee1 = (int *)zalloc((size_t)ne * 3 * 4);
  s->ee2 = (int *)zalloc((size_t)ne * 3 * 4);
  int ned = 0;
  for (int q = 0; q < 3 * ne;) {
    int r = q + 1;
    while (r < 3 * ne && he[r].a == he[q].a && he[r].b == he[q].b) ++r;
    if (r - q > 2 || he[q].a == he[q].b) {
      snprintf(g_create_err, sizeof g_create_err, "edge %d-%d has %d elements", he[q].a, he[q].b,
               r - q);
      free(he);
      ocst_destroy(s);
      return NULL;
    }
    s->en1[ned] = he[q].a;
    s->en2[ned] = he[q].b;
    s->ee1[ned] = he[q].e;
    s->ee2[ned] = r - q == 2 ? he[q + 1].e : -1;
    ++ned;
    q = r;
  }
  free(he);
  s->ned = ned;
  size_t N = (size_t)nn * 8;
  s->ux = (double *)zalloc(N); s->uy = (double *)zalloc(N);
  s->vx = (double *)zalloc(N); s->vy = (double *)zalloc(N);
  s->m = (double *)zalloc(N); s->minv = (double *)zalloc(N);
  s->fx = (double *)zalloc(N); s->fy = (double *)zalloc(N);
  s->Fx = (double *)zalloc(N); s->Fy = (double *)zalloc(N);
  s->Vx = (double *)zalloc(N); s->Vy = (double *)zalloc(N);
  s->Wn = (double *)zalloc(N); s->Wd = (double *)zalloc(N);
  s->lflag = (unsigned char *)zalloc((size_t)nn);
  s->dmask = (unsigned char *)zalloc((size_t)nn);
  s->eps_e = (double *)zalloc((size_t)ne * 3 * 8);
  s->eps_g = (double *)zalloc((size_t)ned * 3 * 8);
  s->sig_g = (double *)zalloc((size_t)ned * 3 * 8);
  s->reccap = 64;
  s->erec = (double *)zalloc((size_t)s->reccap * 7 * 8);
  s->gc = (float *)zalloc((size_t)ne * 4);
  for (int e = 0; e < ne; ++e) s->gc[e] = 3.0f;
  s->gamma = 1.0;
  return s;
}

int ocst_set_fracture(ocst *s, const float *gc, double gc_uniform, double gamma, int gamma_mode) {
  if (gamma_mode < 0 || gamma_mode > 1) return fail(s, -1, "bad gamma mode");
  for (int e = 0; e < s->ne; ++e) s->gc[e] = gc ? gc[e] : (float)gc_uniform;
  s->gamma = gamma;
  s->gamma_mode = gamma_mode;
  return 0;
}

int ocst_n_edges(const ocst *s) { return s->ned; }

int ocst_edges(const ocst *s, int *n1, int *n2, int *e1, int *e2) {
  for (int g = 0; g < s->ned; ++g) {
    if (n1) n1[g] = s->en1[g];
    if (n2) n2[g] = s->en2[g];
    if (e1) e1[g] = s->ee1[g];
    if (e2) e2[g] = s->ee2[g];
  }
  return 0;
}

/* lumped mass: each triangle gives rho A / 3 to each of its nodes, in
 * increasing element id */
int ocst_set_material(ocst *s, double E, double nu, double rho, int plane_strain) {
  if (!(E > 0) || !(nu > -1.0 && nu < 0.5) || !(rho > 0)) return fail(s, -1, "bad material");
  s->E = E; s->nu = nu; s->rho = rho; s->plane_strain = plane_strain != 0;
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
  for (int N = 0; N < s->nn; ++N) s->m[N] = 0.0;
  for (int e = 0; e < s->ne; ++e) {
    double me = (rho * s->A[e]) / 3.0;
    for (int i = 0; i < 3; ++i) s->m[s->conn[3 * e + i]] = s->m[s->conn[3 * e + i]] + me;
  }
  for (int N = 0; N < s->nn; ++N) s->minv[N] = s->m[N] > 0 ? 1.0 / s->m[N] : 0.0;
  s->mat_set = 1;
  if (!s->dt_set) ocst_set_dt(s, 0.5, 0.0);
  return 0;
}

int ocst_set_dt(ocst *s, double dt_factor, double dt_explicit) {
  if (dt_explicit > 0) {
    s->dt = dt_explicit;
  } else {
    if (!s->mat_set) return fail(s, -6, "material first");
    double E = s->E, nu = s->nu, rho = s->rho, cd;
    if (s->plane_strain) cd = sqrt((E * (1.0 - nu)) / (rho * ((1.0 + nu) * (1.0 - 2.0 * nu))));
    else cd = sqrt(E / (rho * (1.0 - nu * nu)));
    s->dt = dt_factor * s->hmin / cd;
  }
  s->dt_set = 1;
  return 0;
}

double ocst_dt(const ocst *s) { return s->dt; }

int ocst_set_energy_every(ocst *s, int K) {
  s->energy_every = K > 0 ? K : 0;
  return 0;
}

static double law_eval(int law, double t, double t0, double tau) {
  if (law == 0) return 1.0;
  if (t <= t0) return t / t0;
  if (law == 1) return 1.0;
  return exp(-(t - t0) / tau);
}

/* outward unit normal and length of boundary edge g, from its element's
 * counter-clockwise order */
static void edge_outward(const ocst *s, int g, double *nx, double *ny, double *L) {
  int e = s->ee1[g];
  int a = -1, b = -1;
  for (int k = 0; k < 3; ++k) {
    int p = s->conn[3 * e + k], q = s->conn[3 * e + (k + 1) % 3];
    if ((p == s->en1[g] && q == s->en2[g]) || (p == s->en2[g] && q == s->en1[g])) { a = p; b = q; }
  }
  double dx = s->X[2 * b] - s->X[2 * a], dy = s->X[2 * b + 1] - s->X[2 * a + 1];
  *L = sqrt(dx * dx + dy * dy);
  *nx = dy / *L;
  *ny = -dx / *L;
}

/* Neumann loads: each node of a loaded edge of length L gets L/2 times the
 * traction, edges in increasing id; prescribed velocities as in the Q4
 * oracle. */
int ocst_add_bc(ocst *s, int kind, int n, const int *items, int comp_mask, int law, double a0,
                double t0, double tau) {
  if (n < 0 || (n > 0 && !items)) return fail(s, -1, "bad items");
  if (law < 0 || law > 2) return fail(s, -1, "bad law");
  if (law != 0 && !(t0 > 0)) return fail(s, -1, "t0 must be > 0");
  if (law == 2 && !(tau > 0)) return fail(s, -1, "tau must be > 0");
  if (kind == 0 || kind == 1) {
    if (s->neu_set && (s->neu_law != law || s->neu_t0 != t0 || s->neu_tau != tau))
      return fail(s, -1, "all Neumann loads share one time law");
    for (int q = 0; q < n; ++q)
      if (items[q] < 0 || items[q] >= s->ned || s->ee2[items[q]] >= 0)
        return fail(s, -1, "edge %d is not a boundary edge", items[q]);
    int *sorted = (int *)zalloc((size_t)n * 4);
    memcpy(sorted, items, (size_t)n * 4);
    for (int a = 1; a < n; ++a) {
      int v = sorted[a], b = a - 1;
      while (b >= 0 && sorted[b] > v) { sorted[b + 1] = sorted[b]; --b; }
      sorted[b + 1] = v;
    }
    for (int q = 0; q < n; ++q) {
      int g = sorted[q];
      double ox, oy, L, tx, ty;
      edge_outward(s, g, &ox, &oy, &L);
      if (kind == 0) {
        tx = (comp_mask & 1) ? a0 : 0.0;
        ty = (comp_mask & 2) ? a0 : 0.0;
      } else { /* pressure pushes into the material */
        tx = -a0 * ox;
        ty = -a0 * oy;
      }
      double half = 0.5 * L;
      int n1 = s->en1[g], n2 = s->en2[g];
      s->Fx[n1] = s->Fx[n1] + half * tx; s->Fy[n1] = s->Fy[n1] + half * ty;
      s->Fx[n2] = s->Fx[n2] + half * tx; s->Fy[n2] = s->Fy[n2] + half * ty;
      s->lflag[n1] = 1; s->lflag[n2] = 1;
    }
    free(sorted);
    s->neu_set = 1; s->neu_law = law; s->neu_t0 = t0; s->neu_tau = tau;
    return 0;
  }
  if (kind == 2) {
    if (s->dir_set && (s->dir_law != law || s->dir_t0 != t0 || s->dir_tau != tau))
      return fail(s, -1, "all Dirichlet loads share one time law");
    if ((comp_mask & 3) == 0) return fail(s, -1, "empty component mask");
    for (int q = 0; q < n; ++q)
      if (items[q] < 0 || items[q] >= s->nn) return fail(s, -1, "bad node %d", items[q]);
    for (int q = 0; q < n; ++q) {
      int N = items[q];
      if (comp_mask & 1) { s->dmask[N] |= 1; s->Vx[N] = a0; }
      if (comp_mask & 2) { s->dmask[N] |= 2; s->Vy[N] = a0; }
    }
    s->dir_set = 1; s->dir_law = law; s->dir_t0 = t0; s->dir_tau = tau;
    return 0;
  }
  return fail(s, -1, "bad kind");
}

int ocst_set_state(ocst *s, const double *ux, const double *uy, const double *vx,
                   const double *vy) {
  if (s->step != 0) return fail(s, -6, "state can only be set before the first step");
  for (int N = 0; N < s->nn; ++N) {
    if (ux) s->ux[N] = ux[N];
    if (uy) s->uy[N] = uy[N];
    if (vx) s->vx[N] = vx[N];
    if (vy) s->vy[N] = vy[N];
  }
  return 0;
}

/* steps 1-4 of the header */
static void compute_forces(ocst *s) {
  /* 1. element strains (exx, eyy, gxy), sums over local nodes 0, 1, 2 */
  for (int e = 0; e < s->ne; ++e) {
    const int *n = s->conn + 3 * e;
    const double *b = s->b + 3 * e, *c = s->c + 3 * e;
    double exx = 0.0, eyy = 0.0, gxy = 0.0;
    for (int i = 0; i < 3; ++i) {
      exx = exx + b[i] * s->ux[n[i]];
      eyy = eyy + c[i] * s->uy[n[i]];
      gxy = gxy + (c[i] * s->ux[n[i]] + b[i] * s->uy[n[i]]);
    }
    s->eps_e[3 * e] = exx;
    s->eps_e[3 * e + 1] = eyy;
    s->eps_e[3 * e + 2] = gxy;
  }
  for (int N = 0; N < s->nn; ++N) { s->fx[N] = 0.0; s->fy[N] = 0.0; }
  for (int g = 0; g < s->ned; ++g) {
    int e1 = s->ee1[g], e2 = s->ee2[g];
    double *ep = s->eps_g + 3 * g, *sg = s->sig_g + 3 * g;
    /* 2. edge strain */
    if (e2 >= 0) {
      double A1 = s->A[e1], A2 = s->A[e2];
      double w1 = A1 / (A1 + A2), w2 = A2 / (A1 + A2);
      for (int q = 0; q < 3; ++q) ep[q] = w1 * s->eps_e[3 * e1 + q] + w2 * s->eps_e[3 * e2 + q];
    } else {
      for (int q = 0; q < 3; ++q) ep[q] = s->eps_e[3 * e1 + q];
    }
    /* 3. stress */
    sg[0] = s->D11 * ep[0] + s->D12 * ep[1];
    sg[1] = s->D12 * ep[0] + s->D11 * ep[1];
    sg[2] = s->D33 * ep[2];
    /* 4. B_j^T sigma A_j / 3 to the nodes of each element of the edge */
    for (int side = 0; side < 2; ++side) {
      int e = side ? e2 : e1;
      if (e < 0) continue;
      double q3 = s->A[e] / 3.0;
      for (int i = 0; i < 3; ++i) {
        int N = s->conn[3 * e + i];
        double bi = s->b[3 * e + i], ci = s->c[3 * e + i];
        s->fx[N] = s->fx[N] + (bi * sg[0] + ci * sg[2]) * q3;
        s->fy[N] = s->fy[N] + (ci * sg[1] + bi * sg[2]) * q3;
      }
    }
  }
}

/* strain energy: each edge's smoothing domain holds a third of the area of
 * each of its triangles; SE = sum_g 1/2 a_g eps_g . sigma_g, edges in order */
static double strain_energy(const ocst *s) {
  double se = 0.0;
  for (int g = 0; g < s->ned; ++g) {
    int e1 = s->ee1[g], e2 = s->ee2[g];
    double a = s->A[e1] / 3.0;
    if (e2 >= 0) a = a + s->A[e2] / 3.0;
    const double *ep = s->eps_g + 3 * g, *sg = s->sig_g + 3 * g;
    double d = ep[0] * sg[0] + ep[1] * sg[1] + ep[2] * sg[2];
    se = se + 0.5 * (a * d);
  }
  return se;
}

static void do_step(ocst *s) {
  int n = s->step;
  double dt = s->dt;
  double t = (double)n * dt;
  compute_forces(s);
  int energy = s->energy_every > 0 && n % s->energy_every == 0;
  double Wn_tot = 0.0, Wd_tot = 0.0, KE = 0.0, SE = 0.0;
  if (energy) {
    for (int N = 0; N < s->nn; ++N) { Wn_tot = Wn_tot + s->Wn[N]; Wd_tot = Wd_tot + s->Wd[N]; }
    SE = strain_energy(s);
  }
  double lamN = s->neu_set ? law_eval(s->neu_law, t, s->neu_t0, s->neu_tau) : 0.0;
  double lamD = s->dir_set ? law_eval(s->dir_law, ((double)n + 0.5) * dt, s->dir_t0, s->dir_tau) : 0.0;
  double dtv = n == 0 ? 0.5 * dt : dt;
  for (int N = 0; N < s->nn; ++N) {
    int loaded = s->lflag[N];
    int dm = s->dmask[N];
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
    r[0] = (double)n; r[1] = t; r[2] = KE; r[3] = SE; r[4] = Wn_tot; r[5] = Wd_tot; r[6] = 0.0;
    s->nrec++;
  }
  s->step = n + 1;
}

int ocst_step(ocst *s, int nsteps) {
  if (!s->mat_set) return fail(s, -6, "material first");
  for (int q = 0; q < nsteps; ++q) do_step(s);
  return 0;
}

int ocst_get_nodes(const ocst *s, double *ux, double *uy, double *vx, double *vy, double *m) {
  for (int N = 0; N < s->nn; ++N) {
    if (ux) ux[N] = s->ux[N];
    if (uy) uy[N] = s->uy[N];
    if (vx) vx[N] = s->vx[N];
    if (vy) vy[N] = s->vy[N];
    if (m) m[N] = s->m[N];
  }
  return 0;
}

int ocst_n_energy(const ocst *s) { return s->nrec; }

int ocst_get_energy(const ocst *s, double *rec) {
  memcpy(rec, s->erec, (size_t)s->nrec * 7 * 8);
  return 0;
}

int ocst_internal_force(ocst *s, double *fx, double *fy) {
  if (!s->mat_set) return fail(s, -6, "material first");
  compute_forces(s);
  for (int N = 0; N < s->nn; ++N) { fx[N] = s->fx[N]; fy[N] = s->fy[N]; }
  return 0;
}

int ocst_strain_energy(ocst *s, double *se) {
  if (!s->mat_set) return fail(s, -6, "material first");
  compute_forces(s);
  *se = strain_energy(s);
  return 0;
}

/* ------------------------------------------------------ crack evaluation */

/* Sec. 2.2, CST: the point is the midpoint g0 of local edge k0 of the intact
 * triangle e (nodes N1 = conn[k0], N2 = conn[k0+1], counter-clockwise).
 *   delta_d = (u_N2 - u_N1) H, H = 1 iff |x_N2 - x_N1|^2 > |X_N2 - X_N1|^2;
 *   candidate j: the segment from g0 to the midpoint g of local edge
 *   k = k0 + 1 + j, unit normal n oriented so that n . (X_N2 - X_N1) > 0,
 *   sigma the stress of edge g as the triangle uses it (the smoothed edge
 *   stress), G_j = delta_d . (sigma n) / 2.
 * Decision: candidates with G > G_c(e); one such wins; with two, the path p
 * wins if G_p > gamma (G_p - G_q) (ratio mode: G_p > gamma G_q), the larger G
 * (the lower local edge on a tie) when both pass, none when neither does. */
int ocst_eval_surface(ocst *s, int n, const int *edge, const int *elem, double *G, int *choice) {
  if (!s->mat_set) return fail(s, -6, "material first");
  compute_forces(s);
  for (int q = 0; q < n; ++q) {
    const int g0 = edge[q], e = elem[q];
    if (g0 < 0 || g0 >= s->ned || e < 0 || e >= s->ne || (s->ee1[g0] != e && s->ee2[g0] != e))
      return fail(s, -1, "point %d: edge %d is not an edge of element %d", q, g0, e);
    const int *cn = s->conn + 3 * e;
    int k0 = -1;
    for (int k = 0; k < 3; ++k) {
      const int a = cn[k], b = cn[(k + 1) % 3];
      if ((a == s->en1[g0] && b == s->en2[g0]) || (a == s->en2[g0] && b == s->en1[g0])) k0 = k;
    }
    const int N1 = cn[k0], N2 = cn[(k0 + 1) % 3];
    const double X1 = s->X[2 * N1], Y1 = s->X[2 * N1 + 1], X2 = s->X[2 * N2], Y2 = s->X[2 * N2 + 1];
    const double dX = X2 - X1, dY = Y2 - Y1;
    const double dux = s->ux[N2] - s->ux[N1], duy = s->uy[N2] - s->uy[N1];
    const double lx = dX + dux, ly = dY + duy;
    const int H = lx * lx + ly * ly > dX * dX + dY * dY;
    const double ddx = H ? dux : 0.0, ddy = H ? duy : 0.0;
    const double mx0 = 0.5 * (X1 + X2), my0 = 0.5 * (Y1 + Y2);
    double Gj[2];
    int kj[2];
    for (int j = 0; j < 2; ++j) {
      const int k = (k0 + 1 + j) % 3;
      kj[j] = k;
      const int a = cn[k], b = cn[(k + 1) % 3];
      const double mx = 0.5 * (s->X[2 * a] + s->X[2 * b]), my = 0.5 * (s->X[2 * a + 1] + s->X[2 * b + 1]);
      const double tx = mx - mx0, ty = my - my0;
      const double L = sqrt(tx * tx + ty * ty);
      double nx = -ty / L, ny = tx / L;
      if (nx * dX + ny * dY < 0) { nx = -nx; ny = -ny; }
      /* the edge of the triangle's local edge k */
      int g = -1;
      for (int h = 0; h < s->ned; ++h)
        if ((s->en1[h] == (a < b ? a : b)) && (s->en2[h] == (a < b ? b : a))) { g = h; break; }
      const double *sg = s->sig_g + 3 * g;
      const double snx = sg[0] * nx + sg[2] * ny, sny = sg[2] * nx + sg[1] * ny;
      Gj[j] = 0.5 * (ddx * snx + ddy * sny);
      G[2 * q + j] = Gj[j];
    }
    const double gc = (double)s->gc[e];
    const int a0 = Gj[0] > gc, a1 = Gj[1] > gc;
    int pick = -1;
    if (a0 && !a1) pick = 0;
    else if (a1 && !a0) pick = 1;
    else if (a0 && a1) {
      const int p0 = s->gamma_mode ? Gj[0] > s->gamma * Gj[1] : Gj[0] > s->gamma * (Gj[0] - Gj[1]);
      const int p1 = s->gamma_mode ? Gj[1] > s->gamma * Gj[0] : Gj[1] > s->gamma * (Gj[1] - Gj[0]);
      if (p0 && p1) pick = Gj[1] > Gj[0] ? 1 : (Gj[0] > Gj[1] ? 0 : (kj[0] < kj[1] ? 0 : 1));
      else if (p0) pick = 0;
      else if (p1) pick = 1;
    }
    choice[q] = pick < 0 ? -1 : kj[pick];
  }
  return 0;
}
