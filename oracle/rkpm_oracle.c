/*
 * rkpm_oracle.c -- traditional (neighbour-loop) RKPM for the Poisson problem in
 * 3D (and, on grids with trailing axes of one point, in 2D and 1D: Sec. 6.1), in
 * FP64 on the CPU.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the GPU path is checked
 * against.  Only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark may load it; the product path never does.  It shares no code, header,
 * table or constant with the CUDA library: it works on the nodes of the domain
 * only (no periodic box, no FFT, no convolution), with an explicit neighbour
 * search, explicit moment matrices, explicit shape functions and an assembled
 * sparse stiffness matrix, exactly as the traditional method of Sec. 2 does.
 *
 * Index space.  Nodes sit on a uniform grid of n[0] x n[1] x n[2] points with
 * spacing h[k] (x fastest: idx = i + n0*(j + n1*k)).  A grid point is a node of
 * the discretisation iff chi[idx] == 1 (Eq. 40); points with chi == 0 do not
 * exist for this method.  The grid is NOT periodic: a neighbour must lie inside
 * the grid.
 *
 * Readings of the paper used here:
 *  - Eq. 7 at z >= 1 is taken as exactly 0, and its second branch is evaluated
 *    in the factored form (4/3)(1-z)^3 (same polynomial).  A node at distance
 *    exactly a is therefore not a neighbour.
 *  - The monomial basis of Eq. 4 is used in the scaled form H((x - x_I)/a),
 *    i.e. each monomial x^alpha divided by a^|alpha|.  This is the diagonal
 *    change of basis H_s = D H; it leaves Psi (Eq. 2) and the implicit gradient
 *    Psi^grad (Eq. 15) unchanged, and only makes M better conditioned.  With it,
 *    b^0 = first row of M_s^{-1} and b^k = -(1/a_k) * row (1+k) of M_s^{-1}
 *    (Eq. 45-47 rewritten for the scaled basis).
 *  - Basis ordering (Eq. 4 extended to 3D): [1, x, y, z] for n = 1 and
 *    [1, x, y, z, x^2, xy, xz, y^2, yz, z^2] for n = 2; in 2D and 1D the entries
 *    that involve only the present coordinates, in the same order.
 *
 * Parity pins: see the oracle tests (reproducing conditions, closed-form
 * interior stencil at a = 2h, neighbour counts of Tab. 4-5, K symmetry,
 * K.1 = 0, energy of linear fields, manufactured-solution convergence).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXS 10

/* Threads.  Loops over nodes, rows or samples whose iterations are independent
   run on all host threads (OpenMP, when the library is built with it); every
   value is computed by one thread in the same order whatever the thread count,
   and sums across nodes (dot products) add fixed blocks in block order, so the
   results do not depend on the number of threads. */
int orc_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Kernel and basis                                                          */
/* ------------------------------------------------------------------------ */

/* Eq. 7: cubic B-spline profile on one axis, z = |x| / a. */
double orc_phi1(double z) {
  if (z < 0.0) z = -z;
  if (z >= 1.0) return 0.0;
  if (z <= 0.5) return 2.0 / 3.0 - 4.0 * z * z + 4.0 * z * z * z;
  double t = 1.0 - z;
  return (4.0 / 3.0) * t * t * t;
}

/* Eq. 5: number of monomials of degree <= n in 3D. */
int orc_basis_size(int degree) { return degree == 1 ? 4 : (degree == 2 ? 10 : -1); }

/* The same in dim = 1, 2, 3 dimensions: (n + dim)! / (n! dim!). */
int orc_basis_size_dim(int degree, int dim) {
  if (degree != 1 && degree != 2) return -1;
  if (dim == 1) return degree + 1;
  if (dim == 2) return degree == 1 ? 3 : 6;
  if (dim == 3) return orc_basis_size(degree);
  return -1;
}

/* Eq. 4, scaled argument xi = (x - x_I)/a, in dim dimensions.  The paper states
   the method in 2D and obtains 1D and 3D by dropping or adding a coordinate, so
   the monomials are those of the 3D list [1, x, y, z, x^2, xy, xz, y^2, yz, z^2]
   that involve only the first dim coordinates, in that order. */
static void basis(int degree, int dim, const double xi[3], double *H) {
  int q = 0;
  H[q++] = 1.0;
  for (int k = 0; k < dim; ++k) H[q++] = xi[k];
  if (degree == 2)
    for (int k = 0; k < dim; ++k)
      for (int l = k; l < dim; ++l) H[q++] = xi[k] * xi[l];
}

/* ------------------------------------------------------------------------ */
/* Geometry                                                                  */
/* ------------------------------------------------------------------------ */

typedef struct {
  int n[3];
  double h[3];
  double a[3];     /* support size per axis, Eq. 64: a_k = a_tilde * h_k */
  int dim;         /* axes with n[k] > 1; the others (trailing) are absent */
  int degree, s;
  int r[3];        /* reach: largest |offset| with phi1 > 0 on that axis */
  int w[3];        /* 2r+1 */
  int nslot;       /* w0*w1*w2 neighbour slots per evaluation node */
  const uint8_t *chi;
} geom_t;

static int64_t gidx(const geom_t *g, int i, int j, int k) {
  return (int64_t)i + (int64_t)g->n[0] * ((int64_t)j + (int64_t)g->n[1] * k);
}

static void gcoord(const geom_t *g, int64_t idx, int c[3]) {
  c[0] = (int)(idx % g->n[0]);
  c[1] = (int)((idx / g->n[0]) % g->n[1]);
  c[2] = (int)(idx / ((int64_t)g->n[0] * g->n[1]));
}

/* Dimension of a grid: 3, or 2 when n[2] == 1, or 1 when n[1] == n[2] == 1
   (absent axes are trailing); -1 otherwise. */
int orc_grid_dim(const int n[3]) {
  if (n[0] < 2) return -1;
  if (n[1] == 1) return n[2] == 1 ? 1 : -1;
  return n[2] == 1 ? 2 : 3;
}

static int geom_init(geom_t *g, const int n[3], const double h[3], double a_tilde, int degree,
                     const uint8_t *chi) {
  g->degree = degree;
  g->dim = orc_grid_dim(n);
  if (g->dim < 0) return -1;
  g->s = orc_basis_size_dim(degree, g->dim);
  if (g->s < 0) return -1;
  g->nslot = 1;
  for (int k = 0; k < 3; ++k) {
    g->n[k] = n[k];
    g->h[k] = h[k];
    g->a[k] = a_tilde * h[k];
    int r = 0;
    while (k < g->dim && orc_phi1(((double)(r + 1) * h[k]) / g->a[k]) > 0.0) ++r;
    g->r[k] = r;
    g->w[k] = 2 * r + 1;
    g->nslot *= g->w[k];
  }
  g->chi = chi;
  return 0;
}

/* Slot of the neighbour at grid offset o (node I = S + o) around an evaluation node S. */
static int slot_of(const geom_t *g, const int o[3]) {
  return ((o[2] + g->r[2]) * g->w[1] + (o[1] + g->r[1])) * g->w[0] + (o[0] + g->r[0]);
}

static void offset_of(const geom_t *g, int slot, int o[3]) {
  o[0] = slot % g->w[0] - g->r[0];
  o[1] = (slot / g->w[0]) % g->w[1] - g->r[1];
  o[2] = slot / (g->w[0] * g->w[1]) - g->r[2];
}

/* ------------------------------------------------------------------------ */
/* Small dense SPD solve (Cholesky)                                          */
/* ------------------------------------------------------------------------ */

/* In-place Cholesky M = L L^T of an s x s SPD matrix (row-major, lower part used).
   Returns 0, or 1 if a pivot is not positive relative to the trace. */
static int cholesky(int s, double *M) {
  double tr = 0.0;
  for (int i = 0; i < s; ++i) tr += fabs(M[i * s + i]);
  for (int j = 0; j < s; ++j) {
    double d = M[j * s + j];
    for (int k = 0; k < j; ++k) d -= M[j * s + k] * M[j * s + k];
    if (!(d > 1e-14 * tr)) return 1;
    double l = sqrt(d);
    M[j * s + j] = l;
    for (int i = j + 1; i < s; ++i) {
      double v = M[i * s + j];
      for (int k = 0; k < j; ++k) v -= M[i * s + k] * M[j * s + k];
      M[i * s + j] = v / l;
    }
  }
  return 0;
}

/* Solve L L^T x = rhs in place. */
static void chol_solve(int s, const double *L, double *x) {
  for (int i = 0; i < s; ++i) {
    double v = x[i];
    for (int k = 0; k < i; ++k) v -= L[i * s + k] * x[k];
    x[i] = v / L[i * s + i];
  }
  for (int i = s - 1; i >= 0; --i) {
    double v = x[i];
    for (int k = i + 1; k < s; ++k) v -= L[k * s + i] * x[k];
    x[i] = v / L[i * s + i];
  }
}

/* ------------------------------------------------------------------------ */
/* Shape functions at one evaluation node S                                  */
/* ------------------------------------------------------------------------ */

/*
 * For a chi node S: for every neighbour slot, the shape function Psi_I(x_S)
 * (Eq. 2) and the implicit gradients Psi^{grad k}_I(x_S), k = x,y,z (Eq. 15-16),
 * where I = S + offset(slot).  Slots whose node is outside the grid, has chi = 0
 * or lies outside the support get 0.  Also returns b^0, b^x, b^y, b^z at S
 * (4*s values, scaled-basis convention).  Returns 0, or 1 if M(x_S) is singular.
 */
static int shape_at(const geom_t *g, int64_t S, double *psi, double *dpsi, double *bout) {
  const int s = g->s;
  int cS[3];
  gcoord(g, S, cS);
  double M[ORC_MAXS * ORC_MAXS];
  double H[ORC_MAXS];
  memset(M, 0, sizeof(M));
  /* Eq. 3 restricted to existing nodes (Eq. 48 with chi(x_S) = 1) */
  for (int sl = 0; sl < g->nslot; ++sl) {
    int o[3];
    offset_of(g, sl, o);
    int cI[3] = {cS[0] + o[0], cS[1] + o[1], cS[2] + o[2]};
    psi[sl] = 0.0;
    dpsi[3 * sl + 0] = dpsi[3 * sl + 1] = dpsi[3 * sl + 2] = 0.0;
    if (cI[0] < 0 || cI[0] >= g->n[0] || cI[1] < 0 || cI[1] >= g->n[1] || cI[2] < 0 ||
        cI[2] >= g->n[2])
      continue;
    if (!g->chi[gidx(g, cI[0], cI[1], cI[2])]) continue;
    double xi[3] = {0.0, 0.0, 0.0}, ph = 1.0;
    for (int k = 0; k < g->dim; ++k) {  /* Eq. 6: product kernel over the present axes */
      double dx = (double)(cS[k] - cI[k]) * g->h[k]; /* x_S - x_I */
      xi[k] = dx / g->a[k];
      ph *= orc_phi1(fabs(dx) / g->a[k]);
    }
    if (ph == 0.0) continue;
    basis(g->degree, g->dim, xi, H);
    for (int p = 0; p < s; ++p)
      for (int q = 0; q < s; ++q) M[p * s + q] += H[p] * H[q] * ph;
  }
  if (cholesky(s, M)) return 1;
  /* rows 1..1+dim of M^{-1} (M symmetric: row i = M^{-1} e_i) */
  double rows[4][ORC_MAXS];
  memset(rows, 0, sizeof(rows));
  for (int i = 0; i <= g->dim; ++i) {
    for (int p = 0; p < s; ++p) rows[i][p] = (p == i) ? 1.0 : 0.0;
    chol_solve(s, M, rows[i]);
  }
  double b[4][ORC_MAXS];
  for (int p = 0; p < s; ++p) {
    b[0][p] = rows[0][p];                     /* Eq. 45 */
    for (int k = 0; k < 3; ++k)               /* Eq. 46-47; 0 on an absent axis */
      b[1 + k][p] = k < g->dim ? -rows[1 + k][p] / g->a[k] : 0.0;
  }
  if (bout)
    for (int i = 0; i < 4; ++i)
      for (int p = 0; p < s; ++p) bout[i * s + p] = b[i][p];
  /* Eq. 2 and Eq. 15 */
  for (int sl = 0; sl < g->nslot; ++sl) {
    int o[3];
    offset_of(g, sl, o);
    int cI[3] = {cS[0] + o[0], cS[1] + o[1], cS[2] + o[2]};
    if (cI[0] < 0 || cI[0] >= g->n[0] || cI[1] < 0 || cI[1] >= g->n[1] || cI[2] < 0 ||
        cI[2] >= g->n[2])
      continue;
    if (!g->chi[gidx(g, cI[0], cI[1], cI[2])]) continue;
    double xi[3] = {0.0, 0.0, 0.0}, ph = 1.0;
    for (int k = 0; k < g->dim; ++k) {
      double dx = (double)(cS[k] - cI[k]) * g->h[k];
      xi[k] = dx / g->a[k];
      ph *= orc_phi1(fabs(dx) / g->a[k]);
    }
    if (ph == 0.0) continue;
    basis(g->degree, g->dim, xi, H);
    double v0 = 0.0, vx = 0.0, vy = 0.0, vz = 0.0;
    for (int p = 0; p < s; ++p) {
      v0 += b[0][p] * H[p];
      vx += b[1][p] * H[p];
      vy += b[2][p] * H[p];
      vz += b[3][p] * H[p];
    }
    psi[sl] = v0 * ph;
    dpsi[3 * sl + 0] = vx * ph;
    dpsi[3 * sl + 1] = vy * ph;
    dpsi[3 * sl + 2] = vz * ph;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Context: all shape functions of the discretisation                        */
/* ------------------------------------------------------------------------ */

typedef struct {
  geom_t g;
  int64_t nbox;
  int64_t nnode;      /* number of chi nodes */
  int64_t *node_box;  /* box index of each chi node */
  int64_t *box_node;  /* node number of each grid point, -1 if chi == 0 */
  double *psi;        /* nnode * nslot */
  double *dpsi;       /* nnode * nslot * 3 */
  double *b;          /* nnode * 4 * s */
  int64_t nsingular;
  int64_t first_singular; /* box index, -1 if none */
  uint8_t *chi_copy;
  /* assembled stiffness (CSR over node numbers), built on demand */
  int64_t *kptr;
  int64_t *kcol;
  double *kval;
} orc_ctx;

void orc_destroy(orc_ctx *c) {
  if (!c) return;
  free(c->node_box);
  free(c->box_node);
  free(c->psi);
  free(c->dpsi);
  free(c->b);
  free(c->chi_copy);
  free(c->kptr);
  free(c->kcol);
  free(c->kval);
  free(c);
}

/* Build all shape functions.  Returns NULL on allocation failure or bad degree. */
orc_ctx *orc_create(const int n[3], const double h[3], double a_tilde, int degree,
                    const uint8_t *chi) {
  orc_ctx *c = (orc_ctx *)calloc(1, sizeof(orc_ctx));
  if (!c) return NULL;
  c->nbox = (int64_t)n[0] * n[1] * n[2];
  c->chi_copy = (uint8_t *)malloc((size_t)c->nbox);
  if (!c->chi_copy) { orc_destroy(c); return NULL; }
  for (int64_t i = 0; i < c->nbox; ++i) c->chi_copy[i] = chi[i] ? 1 : 0;
  if (geom_init(&c->g, n, h, a_tilde, degree, c->chi_copy)) { orc_destroy(c); return NULL; }
  c->box_node = (int64_t *)malloc(sizeof(int64_t) * (size_t)c->nbox);
  if (!c->box_node) { orc_destroy(c); return NULL; }
  c->nnode = 0;
  for (int64_t i = 0; i < c->nbox; ++i) c->box_node[i] = c->chi_copy[i] ? c->nnode++ : -1;
  c->node_box = (int64_t *)malloc(sizeof(int64_t) * (size_t)(c->nnode + 1));
  c->psi = (double *)malloc(sizeof(double) * (size_t)(c->nnode * c->g.nslot + 1));
  c->dpsi = (double *)malloc(sizeof(double) * (size_t)(c->nnode * c->g.nslot * 3 + 1));
  c->b = (double *)malloc(sizeof(double) * (size_t)(c->nnode * 4 * c->g.s + 1));
  if (!c->node_box || !c->psi || !c->dpsi || !c->b) { orc_destroy(c); return NULL; }
  for (int64_t i = 0; i < c->nbox; ++i)
    if (c->box_node[i] >= 0) c->node_box[c->box_node[i]] = i;
  c->nsingular = 0;
  c->first_singular = -1;
  uint8_t *bad = (uint8_t *)calloc((size_t)c->nnode + 1, 1);
  if (!bad) { orc_destroy(c); return NULL; }
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t S = 0; S < c->nnode; ++S) {
    bad[S] = (uint8_t)shape_at(&c->g, c->node_box[S], c->psi + S * c->g.nslot,
                               c->dpsi + S * c->g.nslot * 3, c->b + S * 4 * c->g.s);
    if (bad[S]) {
      memset(c->psi + S * c->g.nslot, 0, sizeof(double) * c->g.nslot);
      memset(c->dpsi + S * c->g.nslot * 3, 0, sizeof(double) * c->g.nslot * 3);
      memset(c->b + S * 4 * c->g.s, 0, sizeof(double) * 4 * c->g.s);
    }
  }
  for (int64_t S = 0; S < c->nnode; ++S)
    if (bad[S]) {
      if (c->first_singular < 0) c->first_singular = c->node_box[S];
      c->nsingular++;
    }
  free(bad);
  return c;
}

int64_t orc_nnode(const orc_ctx *c) { return c->nnode; }
int orc_nslot(const orc_ctx *c) { return c->g.nslot; }
int orc_reach(const orc_ctx *c, int axis) { return c->g.r[axis]; }
int orc_s(const orc_ctx *c) { return c->g.s; }
int orc_dim(const orc_ctx *c) { return c->g.dim; }
int64_t orc_nsingular(const orc_ctx *c) { return c->nsingular; }
int64_t orc_first_singular(const orc_ctx *c) { return c->first_singular; }

/* Node list (box index of each chi node). */
void orc_node_box(const orc_ctx *c, int64_t *out) {
  memcpy(out, c->node_box, sizeof(int64_t) * (size_t)c->nnode);
}

/* Shape-function tables: for evaluation node S (node number) and slot sl the
   neighbour node number (or -1), Psi and the three implicit gradients.  Every
   slot lies within the reach on each axis, so phi > 0 there: a slot inside the
   grid with chi == 1 is a neighbour. */
static int64_t nbr_node(const orc_ctx *c, int64_t S, int sl);
void orc_shape_tables(const orc_ctx *c, int64_t *nbr, double *psi, double *dpsi) {
  const int ns = c->g.nslot;
  for (int64_t S = 0; S < c->nnode; ++S)
    for (int sl = 0; sl < ns; ++sl) {
      nbr[S * ns + sl] = nbr_node(c, S, sl);
      psi[S * ns + sl] = c->psi[S * ns + sl];
      for (int k = 0; k < 3; ++k) dpsi[(S * ns + sl) * 3 + k] = c->dpsi[(S * ns + sl) * 3 + k];
    }
}

/* Number of neighbours of node S found by the grid search (slots with a node). */
int orc_neighbour_count(const orc_ctx *c, int64_t S) {
  const geom_t *g = &c->g;
  int cS[3], cnt = 0;
  gcoord(g, c->node_box[S], cS);
  for (int sl = 0; sl < g->nslot; ++sl) {
    int o[3];
    offset_of(g, sl, o);
    int cI[3] = {cS[0] + o[0], cS[1] + o[1], cS[2] + o[2]};
    if (cI[0] < 0 || cI[0] >= g->n[0] || cI[1] < 0 || cI[1] >= g->n[1] || cI[2] < 0 || cI[2] >= g->n[2])
      continue;
    if (!g->chi[gidx(g, cI[0], cI[1], cI[2])]) continue;
    double ph = 1.0;
    for (int k = 0; k < 3; ++k) ph *= orc_phi1(fabs((double)o[k] * g->h[k]) / g->a[k]);
    if (ph > 0.0) ++cnt;
  }
  return cnt;
}

/* Brute-force neighbour count: all chi nodes of the grid, O(N) per node. */
int orc_neighbour_count_bruteforce(const orc_ctx *c, int64_t S) {
  const geom_t *g = &c->g;
  int cS[3], cnt = 0;
  gcoord(g, c->node_box[S], cS);
  for (int64_t I = 0; I < c->nnode; ++I) {
    int cI[3];
    gcoord(g, c->node_box[I], cI);
    double ph = 1.0;
    for (int k = 0; k < 3; ++k) ph *= orc_phi1(fabs((double)(cS[k] - cI[k]) * g->h[k]) / g->a[k]);
    if (ph > 0.0) ++cnt;
  }
  return cnt;
}

/* Correction coefficients on the grid: out[(i*s + p)*nbox + idx] for i in
   {b^0, b^x, b^y, b^z}; 0 where chi == 0. */
void orc_b_fields(const orc_ctx *c, double *out) {
  const int s = c->g.s;
  memset(out, 0, sizeof(double) * (size_t)(4 * s) * (size_t)c->nbox);
  for (int64_t S = 0; S < c->nnode; ++S)
    for (int i = 0; i < 4 * s; ++i) out[(int64_t)i * c->nbox + c->node_box[S]] = c->b[S * 4 * s + i];
}

/* ------------------------------------------------------------------------ */
/* Operators on grid-indexed arrays (values off chi are ignored / set to 0)  */
/* ------------------------------------------------------------------------ */

/* neighbour node number of slot sl around evaluation node S, or -1 */
static int64_t nbr_node(const orc_ctx *c, int64_t S, int sl) {
  const geom_t *g = &c->g;
  int cS[3], o[3];
  gcoord(g, c->node_box[S], cS);
  offset_of(g, sl, o);
  int cI[3] = {cS[0] + o[0], cS[1] + o[1], cS[2] + o[2]};
  if (cI[0] < 0 || cI[0] >= g->n[0] || cI[1] < 0 || cI[1] >= g->n[1] || cI[2] < 0 || cI[2] >= g->n[2])
    return -1;
  return c->box_node[gidx(g, cI[0], cI[1], cI[2])];
}

/* Evaluation node S = I + sigma whose support holds node I (I sits in slot
   -sigma of S), for the slot of offset sigma; -1 if there is none. */
static int64_t covering_node(const orc_ctx *c, int64_t I, int sl, int *slot_of_I) {
  const geom_t *g = &c->g;
  int cI[3], sig[3];
  gcoord(g, c->node_box[I], cI);
  offset_of(g, sl, sig);
  int cS[3] = {cI[0] + sig[0], cI[1] + sig[1], cI[2] + sig[2]};
  if (cS[0] < 0 || cS[0] >= g->n[0] || cS[1] < 0 || cS[1] >= g->n[1] || cS[2] < 0 || cS[2] >= g->n[2])
    return -1;
  int msig[3] = {-sig[0], -sig[1], -sig[2]};
  *slot_of_I = slot_of(g, msig);
  return c->box_node[gidx(g, cS[0], cS[1], cS[2])];
}

/* Eq. 50 with direct nodal integration (Eq. 54), matrix-free, both sums written
   as gathers: g^k_S = sum_J Psi^{grad k}_J(x_S) d_J at every evaluation node S,
   then f_I = sum_S V_S sum_k Psi^{grad k}_I(x_S) g^k_S over the S whose support
   holds I. */
void orc_apply_K(const orc_ctx *c, const double *V, const double *d, double *f) {
  const int ns = c->g.nslot;
  double *G = (double *)malloc(sizeof(double) * (size_t)(3 * c->nnode + 1));
  if (!G) {
    for (int64_t i = 0; i < c->nbox; ++i) f[i] = NAN;
    return;
  }
#pragma omp parallel for schedule(static)
  for (int64_t S = 0; S < c->nnode; ++S) {
    double gk[3] = {0.0, 0.0, 0.0};
    const double *dp = c->dpsi + S * ns * 3;
    for (int sl = 0; sl < ns; ++sl) {
      int64_t J = nbr_node(c, S, sl);
      if (J < 0) continue;
      double dJ = d[c->node_box[J]];
      gk[0] += dp[3 * sl + 0] * dJ;
      gk[1] += dp[3 * sl + 1] * dJ;
      gk[2] += dp[3 * sl + 2] * dJ;
    }
    G[3 * S + 0] = gk[0];
    G[3 * S + 1] = gk[1];
    G[3 * S + 2] = gk[2];
  }
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < c->nbox; ++i) f[i] = 0.0;
#pragma omp parallel for schedule(static)
  for (int64_t I = 0; I < c->nnode; ++I) {
    double acc = 0.0;
    for (int sl = 0; sl < ns; ++sl) {
      int tI;
      int64_t S = covering_node(c, I, sl, &tI);
      if (S < 0) continue;
      const double *dI = c->dpsi + (S * ns + tI) * 3;
      acc += V[c->node_box[S]] * (dI[0] * G[3 * S + 0] + dI[1] * G[3 * S + 1] + dI[2] * G[3 * S + 2]);
    }
    f[c->node_box[I]] = acc;
  }
  free(G);
}

/* Eq. 27 with direct nodal integration (Eq. 59): f^r_I = sum_S V_S Psi_I(x_S) r_S,
   gathered over the S whose support holds I. */
void orc_rhs(const orc_ctx *c, const double *V, const double *r, double *fr) {
  const int ns = c->g.nslot;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < c->nbox; ++i) fr[i] = 0.0;
#pragma omp parallel for schedule(static)
  for (int64_t I = 0; I < c->nnode; ++I) {
    double acc = 0.0;
    for (int sl = 0; sl < ns; ++sl) {
      int tI;
      int64_t S = covering_node(c, I, sl, &tI);
      if (S < 0) continue;
      acc += c->psi[S * ns + tI] * (V[c->node_box[S]] * r[c->node_box[S]]);
    }
    fr[c->node_box[I]] = acc;
  }
}

/* Eq. 62: u^h(x_I) = sum_J Psi_J(x_I) d_J at every node. */
void orc_eval_u(const orc_ctx *c, const double *d, double *u) {
  const int ns = c->g.nslot;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < c->nbox; ++i) u[i] = 0.0;
#pragma omp parallel for schedule(static)
  for (int64_t S = 0; S < c->nnode; ++S) {
    const double *ps = c->psi + S * ns;
    double v = 0.0;
    for (int sl = 0; sl < ns; ++sl) {
      int64_t J = nbr_node(c, S, sl);
      if (J < 0) continue;
      v += ps[sl] * d[c->node_box[J]];
    }
    u[c->node_box[S]] = v;
  }
}

/*
 * Eq. 1-2 at arbitrary points of a 1D grid: u^h(x) = sum_I Psi_I(x) d_I with
 * Psi_I(x) = b(x)^T H((x - x_I)/a) phi(|x - x_I|/a) and M(x) of Eq. 3 summed over
 * the chi nodes I within the support (x measured from grid node 0, node i at i h).
 * Used for the Gauss-quadrature L2 error of Eq. 100.  Returns the number of points
 * whose M(x) was singular (their value is 0), or -1 if the grid is not 1D.
 */
int64_t orc_eval_points_1d(const orc_ctx *c, int64_t npts, const double *x, const double *d, double *u) {
  const geom_t *g = &c->g;
  if (g->dim != 1) return -1;
  const int s = g->s;
  const double h = g->h[0], a = g->a[0];
  int64_t bad = 0;
  for (int64_t q = 0; q < npts; ++q) {
    u[q] = 0.0;
    const int i0 = (int)floor(x[q] / h);
    double M[ORC_MAXS * ORC_MAXS], H[ORC_MAXS];
    memset(M, 0, sizeof(M));
    for (int i = i0 - g->r[0] - 1; i <= i0 + g->r[0] + 1; ++i) {
      if (i < 0 || i >= g->n[0] || !g->chi[i]) continue;
      const double xi[3] = {(x[q] - i * h) / a, 0.0, 0.0};
      const double ph = orc_phi1(fabs(xi[0]));
      if (ph == 0.0) continue;
      basis(g->degree, 1, xi, H);
      for (int p = 0; p < s; ++p)
        for (int r = 0; r < s; ++r) M[p * s + r] += H[p] * H[r] * ph;
    }
    if (cholesky(s, M)) { ++bad; continue; }
    double b0[ORC_MAXS];
    for (int p = 0; p < s; ++p) b0[p] = p == 0 ? 1.0 : 0.0;
    chol_solve(s, M, b0); /* first row of M^{-1} (Eq. 45) */
    double v = 0.0;
    for (int i = i0 - g->r[0] - 1; i <= i0 + g->r[0] + 1; ++i) {
      if (i < 0 || i >= g->n[0] || !g->chi[i]) continue;
      const double xi[3] = {(x[q] - i * h) / a, 0.0, 0.0};
      const double ph = orc_phi1(fabs(xi[0]));
      if (ph == 0.0) continue;
      basis(g->degree, 1, xi, H);
      double psi = 0.0;
      for (int p = 0; p < s; ++p) psi += b0[p] * H[p];
      v += psi * ph * d[i];
    }
    u[q] = v;
  }
  return bad;
}

/* Transpose of Eq. 62: w_J = sum_I Psi_J(x_I) e_I, gathered over the nodes I
   whose support holds J. */
void orc_eval_u_transpose(const orc_ctx *c, const double *e, double *w) {
  const int ns = c->g.nslot;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < c->nbox; ++i) w[i] = 0.0;
#pragma omp parallel for schedule(static)
  for (int64_t J = 0; J < c->nnode; ++J) {
    double acc = 0.0;
    for (int sl = 0; sl < ns; ++sl) {
      int tJ;
      int64_t I = covering_node(c, J, sl, &tJ);
      if (I < 0) continue;
      acc += c->psi[I * ns + tJ] * e[c->node_box[I]];
    }
    w[c->node_box[J]] = acc;
  }
}

/* Gradient-type nonlinear force (Eq. B.6-B.8 with DNI): f_J = sum_S V_S sum_k
   Psi^{grad k}_J(x_S) N^k_S over the quadrature nodes S whose support holds J,
   i.e. B^T applied to the field of vectors N (three box fields, N^k at offset
   k*nbox; V box-indexed).  Gathered per J; zero outside chi. */
void orc_grad_transpose(const orc_ctx *c, const double *V, const double *N, double *f) {
  const int ns = c->g.nslot;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < c->nbox; ++i) f[i] = 0.0;
#pragma omp parallel for schedule(static)
  for (int64_t J = 0; J < c->nnode; ++J) {
    double acc = 0.0;
    for (int sl = 0; sl < ns; ++sl) {
      int tJ;
      const int64_t S = covering_node(c, J, sl, &tJ);
      if (S < 0) continue;
      const int64_t bs = c->node_box[S];
      const double *g = c->dpsi + ((size_t)S * ns + tJ) * 3;
      acc += V[bs] * (g[0] * N[bs] + g[1] * N[c->nbox + bs] + g[2] * N[2 * c->nbox + bs]);
    }
    f[c->node_box[J]] = acc;
  }
}

/* ------------------------------------------------------------------------ */
/* Assembled stiffness matrix (Eq. 26 with DNI), CSR over node numbers       */
/* ------------------------------------------------------------------------ */

/* Row I of K (Eq. 26 with DNI): K_IJ = sum_S V_S sum_k Psi^{grad k}_I(x_S)
   Psi^{grad k}_J(x_S) over the quadrature nodes S whose support holds I, each
   pair (I, J) accumulated in a local window of offsets J - I; the nonzeros are
   appended to (*col, *val) in window order.  Returns 0, or -1 on allocation
   failure. */
typedef struct {
  int64_t n, cap;
  int64_t *col;
  double *val;
} orc_rowbuf;

static int assemble_row(const orc_ctx *c, const double *V, int64_t I, double *acc, uint8_t *hit, orc_rowbuf *rb) {
  const geom_t *g = &c->g;
  const int ns = g->nslot;
  const int W[3] = {4 * g->r[0] + 1, 4 * g->r[1] + 1, 4 * g->r[2] + 1};
  const int64_t nloc = (int64_t)W[0] * W[1] * W[2];
  int cI[3];
  gcoord(g, c->node_box[I], cI);
  /* quadrature nodes S whose support covers I: S = I + sigma, and I sits in
     slot (-sigma) of S */
  for (int sl = 0; sl < ns; ++sl) {
    int sig[3];
    offset_of(g, sl, sig);
    int cS[3] = {cI[0] + sig[0], cI[1] + sig[1], cI[2] + sig[2]};
    if (cS[0] < 0 || cS[0] >= g->n[0] || cS[1] < 0 || cS[1] >= g->n[1] || cS[2] < 0 || cS[2] >= g->n[2])
      continue;
    int64_t S = c->box_node[gidx(g, cS[0], cS[1], cS[2])];
    if (S < 0) continue;
    int msig[3] = {-sig[0], -sig[1], -sig[2]};
    const double *dI = c->dpsi + (S * ns + slot_of(g, msig)) * 3;
    if (dI[0] == 0.0 && dI[1] == 0.0 && dI[2] == 0.0) continue;
    double VS = V[c->node_box[S]];
    for (int tl = 0; tl < ns; ++tl) {
      int64_t J = nbr_node(c, S, tl);
      if (J < 0) continue;
      int tau[3];
      offset_of(g, tl, tau);
      const double *dJ = c->dpsi + (S * ns + tl) * 3;
      int64_t li = ((int64_t)(sig[2] + tau[2] + 2 * g->r[2]) * W[1] + (sig[1] + tau[1] + 2 * g->r[1])) * W[0] +
                   (sig[0] + tau[0] + 2 * g->r[0]);
      acc[li] += VS * (dI[0] * dJ[0] + dI[1] * dJ[1] + dI[2] * dJ[2]);
      hit[li] = 1;
    }
  }
  for (int64_t li = 0; li < nloc; ++li) {
    if (!hit[li]) continue;
    int o[3] = {(int)(li % W[0]) - 2 * g->r[0], (int)((li / W[0]) % W[1]) - 2 * g->r[1],
                (int)(li / ((int64_t)W[0] * W[1])) - 2 * g->r[2]};
    int cJ[3] = {cI[0] + o[0], cI[1] + o[1], cI[2] + o[2]};
    int64_t J = c->box_node[gidx(g, cJ[0], cJ[1], cJ[2])];
    if (rb->n >= rb->cap) {
      int64_t ncap = rb->cap * 2 + 1024;
      int64_t *nc = (int64_t *)realloc(rb->col, sizeof(int64_t) * (size_t)ncap);
      if (nc) rb->col = nc;
      double *nv = (double *)realloc(rb->val, sizeof(double) * (size_t)ncap);
      if (nv) rb->val = nv;
      if (!nc || !nv) return -1;
      rb->cap = ncap;
    }
    rb->col[rb->n] = J;
    rb->val[rb->n] = acc[li];
    ++rb->n;
    acc[li] = 0.0;
    hit[li] = 0;
  }
  return 0;
}

/* Assemble K as CSR over node numbers: contiguous blocks of rows per thread,
   concatenated in row order.  Returns the number of nonzeros, or -1 on
   allocation failure. */
int64_t orc_assemble_K(orc_ctx *c, const double *V) {
  const geom_t *g = &c->g;
  const int64_t nloc = (int64_t)(4 * g->r[0] + 1) * (4 * g->r[1] + 1) * (4 * g->r[2] + 1);
  free(c->kptr);
  free(c->kcol);
  free(c->kval);
  c->kcol = NULL;
  c->kval = NULL;
  c->kptr = (int64_t *)malloc(sizeof(int64_t) * (size_t)(c->nnode + 1));
  if (!c->kptr) return -1;
  const int nt = orc_threads();
  orc_rowbuf *rb = (orc_rowbuf *)calloc((size_t)nt, sizeof(orc_rowbuf));
  if (!rb) return -1;
  int failed = 0;
#pragma omp parallel num_threads(nt)
  {
#ifdef _OPENMP
    const int t = omp_get_thread_num(), nth = omp_get_num_threads();
#else
    const int t = 0, nth = 1;
#endif
    const int64_t lo = c->nnode * t / nth, hi = c->nnode * (t + 1) / nth;
    double *acc = (double *)calloc((size_t)nloc, sizeof(double));
    uint8_t *hit = (uint8_t *)calloc((size_t)nloc, 1);
    if (!acc || !hit) {
#pragma omp atomic write
      failed = 1;
    } else {
      for (int64_t I = lo; I < hi; ++I) {
        if (assemble_row(c, V, I, acc, hit, &rb[t])) {
#pragma omp atomic write
          failed = 1;
          break;
        }
        c->kptr[I + 1] = rb[t].n;  /* row end within this thread's block, offset below */
      }
    }
    free(acc);
    free(hit);
  }
  int64_t nnz = 0;
  if (!failed) {
    for (int t = 0; t < nt; ++t) nnz += rb[t].n;
    c->kcol = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nnz + 1));
    c->kval = (double *)malloc(sizeof(double) * (size_t)(nnz + 1));
    if (!c->kcol || !c->kval) failed = 1;
  }
  if (!failed) {
    int64_t off = 0;
    c->kptr[0] = 0;
    for (int t = 0; t < nt; ++t) {
      const int64_t lo = c->nnode * t / nt, hi = c->nnode * (t + 1) / nt;
      for (int64_t I = lo; I < hi; ++I) c->kptr[I + 1] += off;
      memcpy(c->kcol + off, rb[t].col, sizeof(int64_t) * (size_t)rb[t].n);
      memcpy(c->kval + off, rb[t].val, sizeof(double) * (size_t)rb[t].n);
      off += rb[t].n;
    }
  }
  for (int t = 0; t < nt; ++t) {
    free(rb[t].col);
    free(rb[t].val);
  }
  free(rb);
  return failed ? -1 : nnz;
}

void orc_get_K(const orc_ctx *c, int64_t *ptr, int64_t *col, double *val) {
  memcpy(ptr, c->kptr, sizeof(int64_t) * (size_t)(c->nnode + 1));
  memcpy(col, c->kcol, sizeof(int64_t) * (size_t)c->kptr[c->nnode]);
  memcpy(val, c->kval, sizeof(double) * (size_t)c->kptr[c->nnode]);
}

/* ------------------------------------------------------------------------ */
/* Dirichlet solve (Eq. 25, 29): K_OO d_O = f^r_O - K_OG g_G                 */
/* ------------------------------------------------------------------------ */

/* y = K_OO x over free nodes (free[I] = 1), x and y indexed by node number */
static void spmv_free(const orc_ctx *c, const uint8_t *freem, const double *x, double *y) {
#pragma omp parallel for schedule(static)
  for (int64_t I = 0; I < c->nnode; ++I) {
    if (!freem[I]) { y[I] = 0.0; continue; }
    double v = 0.0;
    for (int64_t e = c->kptr[I]; e < c->kptr[I + 1]; ++e)
      if (freem[c->kcol[e]]) v += c->kval[e] * x[c->kcol[e]];
    y[I] = v;
  }
}

/* a . b as the ordered sum of the partial sums of fixed blocks of 4096 entries */
#define ORC_DOT_BLOCK 4096
static double dotn(int64_t n, const double *a, const double *b) {
  const int64_t nb = (n + ORC_DOT_BLOCK - 1) / ORC_DOT_BLOCK;
  double stackp[64];
  double *part = nb <= 64 ? stackp : (double *)malloc(sizeof(double) * (size_t)nb);
  if (!part) return NAN;
#pragma omp parallel for schedule(static)
  for (int64_t blk = 0; blk < nb; ++blk) {
    const int64_t lo = blk * ORC_DOT_BLOCK, hi = lo + ORC_DOT_BLOCK < n ? lo + ORC_DOT_BLOCK : n;
    double s = 0.0;
    for (int64_t i = lo; i < hi; ++i) s += a[i] * b[i];
    part[blk] = s;
  }
  double s = 0.0;
  for (int64_t blk = 0; blk < nb; ++blk) s += part[blk];
  if (part != stackp) free(part);
  return s;
}

/*
 * Solve with strong Dirichlet conditions (Eq. 29): d = g on chi_gamma nodes,
 * K_OO d_O = rhs_O - K_OG g_G on the rest.  The assembled K (orc_assemble_K)
 * must exist.  Dense Cholesky when the free count <= dense_max, else conjugate
 * gradients on the CSR to relative residual tol (at most max_iter iterations).
 * rhs, g, d are grid-indexed.  Returns CG iterations (0 for the dense path),
 * -1 on allocation failure, -2 on a non-positive pivot, -3 if CG did not converge.
 * resid_out receives the final relative residual.
 */
int orc_solve_dirichlet(const orc_ctx *c, const uint8_t *chi_gamma, const double *rhs,
                        const double *g, double tol, int max_iter, int dense_max, double *d,
                        double *resid_out) {
  const int64_t nn = c->nnode;
  uint8_t *freem = (uint8_t *)malloc((size_t)nn + 1);
  double *x = (double *)calloc((size_t)nn + 1, sizeof(double));
  double *b = (double *)calloc((size_t)nn + 1, sizeof(double));
  double *t = (double *)calloc((size_t)nn + 1, sizeof(double));
  if (!freem || !x || !b || !t) { free(freem); free(x); free(b); free(t); return -1; }
  int64_t nfree = 0;
  for (int64_t I = 0; I < nn; ++I) {
    freem[I] = chi_gamma[c->node_box[I]] ? 0 : 1;
    nfree += freem[I];
    x[I] = freem[I] ? 0.0 : g[c->node_box[I]];
  }
  /* b = rhs_O - K_OG g_G */
  for (int64_t I = 0; I < nn; ++I) {
    if (!freem[I]) { b[I] = 0.0; continue; }
    double v = rhs[c->node_box[I]];
    for (int64_t e = c->kptr[I]; e < c->kptr[I + 1]; ++e)
      if (!freem[c->kcol[e]]) v -= c->kval[e] * x[c->kcol[e]];
    b[I] = v;
  }
  int ret = 0;
  double bn = sqrt(dotn(nn, b, b));
  if (nfree <= dense_max) {
    int64_t *fidx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nfree + 1));
    int64_t *pos = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nn + 1));
    double *A = (double *)calloc((size_t)(nfree * nfree + 1), sizeof(double));
    double *y = (double *)calloc((size_t)(nfree + 1), sizeof(double));
    if (!fidx || !pos || !A || !y) {
      free(fidx); free(pos); free(A); free(y);
      ret = -1;
      goto done;
    }
    int64_t m = 0;
    for (int64_t I = 0; I < nn; ++I) { pos[I] = freem[I] ? m : -1; if (freem[I]) fidx[m++] = I; }
    for (int64_t a = 0; a < nfree; ++a) {
      int64_t I = fidx[a];
      for (int64_t e = c->kptr[I]; e < c->kptr[I + 1]; ++e)
        if (freem[c->kcol[e]]) A[a * nfree + pos[c->kcol[e]]] += c->kval[e];
      y[a] = b[I];
    }
    /* dense Cholesky, lower triangle */
    for (int64_t j = 0; j < nfree && ret == 0; ++j) {
      double dj = A[j * nfree + j];
      for (int64_t k = 0; k < j; ++k) dj -= A[j * nfree + k] * A[j * nfree + k];
      if (!(dj > 0.0)) { ret = -2; break; }
      double l = sqrt(dj);
      A[j * nfree + j] = l;
      for (int64_t i = j + 1; i < nfree; ++i) {
        double v = A[i * nfree + j];
        const double *Ai = A + i * nfree, *Aj = A + j * nfree;
        for (int64_t k = 0; k < j; ++k) v -= Ai[k] * Aj[k];
        A[i * nfree + j] = v / l;
      }
    }
    if (ret == 0) {
      for (int64_t i = 0; i < nfree; ++i) {
        double v = y[i];
        for (int64_t k = 0; k < i; ++k) v -= A[i * nfree + k] * y[k];
        y[i] = v / A[i * nfree + i];
      }
      for (int64_t i = nfree - 1; i >= 0; --i) {
        double v = y[i];
        for (int64_t k = i + 1; k < nfree; ++k) v -= A[k * nfree + i] * y[k];
        y[i] = v / A[i * nfree + i];
      }
      for (int64_t a = 0; a < nfree; ++a) x[fidx[a]] = y[a];
    }
    free(fidx); free(pos); free(A); free(y);
  } else {
    /* conjugate gradients on K_OO */
    double *r = (double *)calloc((size_t)nn + 1, sizeof(double));
    double *p = (double *)calloc((size_t)nn + 1, sizeof(double));
    double *xf = (double *)calloc((size_t)nn + 1, sizeof(double));
    if (!r || !p || !xf) { free(r); free(p); free(xf); ret = -1; goto done; }
    for (int64_t I = 0; I < nn; ++I) { r[I] = b[I]; p[I] = b[I]; }
    double rr = dotn(nn, r, r);
    int it = 0;
    ret = -3;
    if (bn == 0.0) ret = 0;
    while (bn > 0.0 && it < max_iter) {
      if (sqrt(rr) <= tol * bn) { ret = it; break; }
      spmv_free(c, freem, p, t);
      double pap = dotn(nn, p, t);
      if (!(pap > 0.0)) { ret = -2; break; }
      double alpha = rr / pap;
#pragma omp parallel for schedule(static)
      for (int64_t I = 0; I < nn; ++I) { xf[I] += alpha * p[I]; r[I] -= alpha * t[I]; }
      double rr2 = dotn(nn, r, r);
      double beta = rr2 / rr;
      rr = rr2;
#pragma omp parallel for schedule(static)
      for (int64_t I = 0; I < nn; ++I) p[I] = r[I] + beta * p[I];
      ++it;
      if (it % 50 == 0) { /* replace the recurrence by the true residual */
        spmv_free(c, freem, xf, t);
#pragma omp parallel for schedule(static)
        for (int64_t I = 0; I < nn; ++I) r[I] = freem[I] ? b[I] - t[I] : 0.0;
        rr = dotn(nn, r, r);
      }
    }
    if (ret == -3 && sqrt(rr) <= tol * bn) ret = it;
    for (int64_t I = 0; I < nn; ++I) if (freem[I]) x[I] = xf[I];
    free(r); free(p); free(xf);
  }
  /* true relative residual of the free equations */
  if (ret >= 0 || ret == -3) {
    spmv_free(c, freem, x, t);
    double s2 = 0.0;
    for (int64_t I = 0; I < nn; ++I) if (freem[I]) { double e = b[I] - t[I]; s2 += e * e; }
    /* t used K_OO only: x on free nodes; x on Gamma is g, already in b */
    if (resid_out) *resid_out = bn > 0.0 ? sqrt(s2) / bn : sqrt(s2);
  }
done:
  for (int64_t i = 0; i < c->nbox; ++i) d[i] = 0.0;
  for (int64_t I = 0; I < nn; ++I) d[c->node_box[I]] = x[I];
  free(freem); free(x); free(b); free(t);
  return ret;
}

/* y = K x for grid-indexed x (all chi nodes), from the assembled CSR */
void orc_spmv(const orc_ctx *c, const double *x, double *y) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < c->nbox; ++i) y[i] = 0.0;
#pragma omp parallel for schedule(static)
  for (int64_t I = 0; I < c->nnode; ++I) {
    double v = 0.0;
    for (int64_t e = c->kptr[I]; e < c->kptr[I + 1]; ++e) v += c->kval[e] * x[c->node_box[c->kcol[e]]];
    y[c->node_box[I]] = v;
  }
}

/* ------------------------------------------------------------------------ */
/* Sampled operators for grids too large to tabulate                         */
/* ------------------------------------------------------------------------ */

/*
 * f_I = (K d)_I for a list of grid points I (chi nodes), computed one by one from
 * the definition (Eq. 50 with DNI) without building tables for the whole grid:
 * for every quadrature node S in the support of I, the shape functions at S are
 * built from scratch.  Returns the number of singular moment matrices met.
 */
int64_t orc_apply_K_sampled(const int n[3], const double h[3], double a_tilde, int degree,
                            const uint8_t *chi, const double *V, const double *d,
                            int64_t nsample, const int64_t *sample, double *out) {
  geom_t g;
  if (geom_init(&g, n, h, a_tilde, degree, chi)) return -1;
  int64_t bad = 0;
  int failed = 0;
#pragma omp parallel reduction(+ : bad)
  {
  double *psi = (double *)malloc(sizeof(double) * (size_t)g.nslot);
  double *dpsi = (double *)malloc(sizeof(double) * (size_t)g.nslot * 3);
  if (!psi || !dpsi) {
#pragma omp atomic write
    failed = 1;
  }
#pragma omp for schedule(dynamic, 1)
  for (int64_t q = 0; q < nsample; ++q) {
    int64_t I = sample[q];
    out[q] = 0.0;
    if (!chi[I] || !psi || !dpsi) continue;
    int cI[3];
    gcoord(&g, I, cI);
    double acc = 0.0;
    for (int sl = 0; sl < g.nslot; ++sl) {
      int sig[3];
      offset_of(&g, sl, sig);
      int cS[3] = {cI[0] + sig[0], cI[1] + sig[1], cI[2] + sig[2]};
      if (cS[0] < 0 || cS[0] >= g.n[0] || cS[1] < 0 || cS[1] >= g.n[1] || cS[2] < 0 || cS[2] >= g.n[2])
        continue;
      int64_t S = gidx(&g, cS[0], cS[1], cS[2]);
      if (!chi[S]) continue;
      if (shape_at(&g, S, psi, dpsi, NULL)) { ++bad; continue; }
      int msig[3] = {-sig[0], -sig[1], -sig[2]};
      const double *dI = dpsi + 3 * slot_of(&g, msig);
      double gk[3] = {0.0, 0.0, 0.0};
      for (int tl = 0; tl < g.nslot; ++tl) {
        int tau[3];
        offset_of(&g, tl, tau);
        int cJ[3] = {cS[0] + tau[0], cS[1] + tau[1], cS[2] + tau[2]};
        if (cJ[0] < 0 || cJ[0] >= g.n[0] || cJ[1] < 0 || cJ[1] >= g.n[1] || cJ[2] < 0 || cJ[2] >= g.n[2])
          continue;
        double dJ = d[gidx(&g, cJ[0], cJ[1], cJ[2])];
        gk[0] += dpsi[3 * tl + 0] * dJ;
        gk[1] += dpsi[3 * tl + 1] * dJ;
        gk[2] += dpsi[3 * tl + 2] * dJ;
      }
      acc += V[S] * (dI[0] * gk[0] + dI[1] * gk[1] + dI[2] * gk[2]);
    }
    out[q] = acc;
  }
  free(psi);
  free(dpsi);
  }
  return failed ? -1 : bad;
}

/*
 * Correction coefficients b (4*s values per sample, order b^0, b^x, b^y, b^z)
 * at a list of grid points, built from scratch.  Points with chi == 0 get the
 * values of M = identity (Eq. 48): b^0 = e_1, b^k = -(1/a_k) e_{1+k}.
 */
int64_t orc_b_sampled(const int n[3], const double h[3], double a_tilde, int degree,
                      const uint8_t *chi, int64_t nsample, const int64_t *sample, double *out) {
  geom_t g;
  if (geom_init(&g, n, h, a_tilde, degree, chi)) return -1;
  int64_t bad = 0;
  int failed = 0;
#pragma omp parallel reduction(+ : bad)
  {
  double *psi = (double *)malloc(sizeof(double) * (size_t)g.nslot);
  double *dpsi = (double *)malloc(sizeof(double) * (size_t)g.nslot * 3);
  if (!psi || !dpsi) {
#pragma omp atomic write
    failed = 1;
  }
#pragma omp for schedule(dynamic, 1)
  for (int64_t q = 0; q < nsample; ++q) {
    double *o = out + q * 4 * g.s;
    if (!psi || !dpsi) continue;
    if (!chi[sample[q]]) {
      for (int i = 0; i < 4 * g.s; ++i) o[i] = 0.0;
      o[0] = 1.0;
      for (int k = 0; k < g.dim; ++k) o[(1 + k) * g.s + 1 + k] = -1.0 / g.a[k];
      continue;
    }
    if (shape_at(&g, sample[q], psi, dpsi, o)) ++bad;
  }
  free(psi);
  free(dpsi);
  }
  return failed ? -1 : bad;
}
