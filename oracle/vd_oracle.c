/*
 * vd_oracle.c -- plain, slow FP64 CPU oracle for 3D Voronoi and power cells.
 *
 * TEST INFRASTRUCTURE. Only the test suite, the package smoke check and the
 * CPU-baseline leg of the benchmark load this library. It shares no code,
 * header, table or helper with the CUDA path and never calls it.
 *
 * What it computes (Sec. 3, Eq. 1): for every site i the cell
 *
 *     K_i = bbox  ∩  { x : |x - p_i|^2 - w_i <= |x - p_j|^2 - w_j,  j != i }
 *
 * written out as clipping the box by one half-space per candidate site, in
 * local coordinates x~ = x - p_i where site j gives the plane
 *
 *     n_j . x~ <= b_j,   n_j = p_j - p_i,   b_j = (|n_j|^2 + w_i - w_j) / 2,
 *
 * whose distance to p_i is b_j / |n_j| = d_ij of Eq. 2.
 *
 * Cell representation and clipping follow the supplementary "Convex cell
 * clipping" section (App. B): half-space equations plus vertices stored as
 * ordered plane-index triplets; a clip classifies every vertex, removes the
 * outside ones one at a time while keeping them adjacent to the hole, keeps
 * the hole boundary as a circular list of plane indices (each consecutive
 * pair (a,b) is a dangling edge on faces a and b) and closes the hole with
 * one new vertex (h,a,b) per boundary pair.
 *
 * Orientation convention: a vertex (a,b,c) is stored so that
 * det(n_a, n_b, n_c) > 0. Every box corner starts that way and a new vertex
 * (a,b,h) inherits it from the removed vertex (a,b,c) it replaces on edge
 * a∩b, so the invariant holds for every vertex in exact arithmetic.
 *
 * Predicate. A vertex v = (a,b,c) with Cramer numerators D1..D3 and
 * denominator D0 = det(n_a,n_b,n_c) lies outside plane h iff
 *     T = n_h . (D1,D2,D3) - b_h * D0 > 0
 * (T = D0 * s_v and D0 > 0 by the orientation invariant). Two modes:
 *   - FP64: T in double with a Shewchuk-style static bound built from the
 *     permanents of the same minors; when |T| is below that bound the sign
 *     is taken exactly instead, in floating-point expansion arithmetic
 *     (Shewchuk 1997: TwoSum, FMA TwoProduct, Grow-Expansion) from the
 *     sites' coordinates and weights, as sign(T) * sign(D0). Every sign is
 *     therefore exact; "exact_resolved" counts the predicates that needed
 *     it, "degenerate" those whose exact value is 0 (outside means > 0).
 *   - exact: inputs on a 2^-20 coordinate / 2^-40 weight grid give integer
 *     plane rows, and T is computed exactly in __int128.
 *
 * Candidates: "brute" clips with every other site in ascending d_ij; "kd"
 * streams sites from a k-d tree (our own, with per-node maximum weight) in
 * ascending lower bound of d_ij and stops once that bound exceeds the
 * isotropic security radius max_v |v~| (the criterion of Sec. 4.2 with the
 * node bound of Sec. 4.2.2), which is valid for any candidate order.
 *
 * Outputs per cell: ascending neighbour list (sites whose plane carries a
 * face of the final cell; box faces are not neighbours), volume and
 * centroid by pyramids over fan-triangulated faces, and the
 * Reynolds-transport gradient of L = sum_i c_i V_i + d_i . g_i with the
 * cell combinatorics held fixed.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef __int128 i128;

#define ORC_OK 0
#define ORC_ERR_ARG -1
#define ORC_ERR_TOPOLOGY -2
#define ORC_ERR_NBR_CAP -3
#define ORC_ERR_GRID -4
#define ORC_ERR_MEM -5

/* statistics slots written to the caller's stats[] array */
enum {
  ST_AMBIGUOUS = 0,   /* predicates whose sign could not be certified     */
  ST_DEGENERATE = 1,  /* exact predicates with T == 0 (or D0 == 0)        */
  ST_ORIENT_FAIL = 2, /* exact mode: a new vertex with D0 <= 0            */
  ST_TOPO_FAIL = 3,   /* hole walk could not reach every outside vertex   */
  ST_CLIPS = 4,       /* clips that removed at least one vertex           */
  ST_TESTS = 5,       /* candidate planes tested against the cell         */
  ST_EMPTY = 6,       /* empty cells                                      */
  ST_FACEWALK_FAIL = 7,
  ST_EXACT = 8,       /* FP64 predicates inside the bound, signed exactly */
  ST_N = 9
};

static const double EPS = 1.1102230246251565e-16; /* 2^-53 */

/* ------------------------------------------------------------------ */
/* planes and vertices                                                 */

typedef struct {
  double n[3];   /* outward normal (not normalised)                    */
  double b;      /* right-hand side                                    */
  double bmag;   /* magnitude bound used by the error bound of b       */
  int64_t site;  /* >= 0: site index; < 0: box face -1-k               */
  int64_t owner; /* the cell's site i (the plane is in its frame)      */
  int64_t N[3];  /* exact mode: integer row                            */
  int64_t B;
} plane_t;

typedef struct {
  int p[3];       /* plane indices, det(n_p0, n_p1, n_p2) > 0          */
  double D[4];    /* Cramer numerators D1, D2, D3 and denominator D0   */
  double P[4];    /* permanents of the magnitude minors, same order    */
  double x[3];    /* position (local coordinates)                      */
  double err;     /* bound on |x - x_exact|_2 (inf if ill-posed)       */
  i128 E[4];      /* exact mode: D1, D2, D3, D0                        */
} vert_t;

typedef struct {
  plane_t* pl;
  int npl, cappl;
  vert_t* v;
  int nv, capv;
  int empty;
  /* scratch for clipping */
  int* out;
  int* removed;
  int* list;
  int caplist;
  vert_t* vtmp;
  int capvtmp;
} cell_t;

typedef struct {
  const float* xyz;
  const float* w;
  int64_t n;
  double lo[3], hi[3];
  int exact;
  /* exact mode integer coordinates */
  int64_t* X;  /* [3n] coordinate * 2^20 */
  int64_t* W;  /* [n]  weight * 2^40     */
  int64_t LO[3], HI[3];
  /* sites with an exact duplicate that beats them (larger weight, then lower
   * index): their cells are empty and their half-spaces are implied by the
   * winner's, so they are never candidates */
  unsigned char* dup_loser;
  /* finite differences: site ov_site at (ov_xyz, ov_w) in FP64 instead of
   * its float32 input (-1: none) */
  int64_t ov_site;
  double ov_xyz[3];
  double ov_w;
} problem_t;

static double site_x(const problem_t* pr, int64_t i, int k) {
  return i == pr->ov_site ? pr->ov_xyz[k] : (double)pr->xyz[3 * i + k];
}
static double site_w(const problem_t* pr, int64_t i) {
  return i == pr->ov_site ? pr->ov_w : (pr->w ? (double)pr->w[i] : 0.0);
}

static double dmax(double a, double b) { return a > b ? a : b; }

static void* xrealloc(void* p, size_t sz) {
  void* q = realloc(p, sz);
  if (!q) {
    fprintf(stderr, "vd_oracle: out of memory\n");
    abort();
  }
  return q;
}

static void cell_init_storage(cell_t* C) {
  memset(C, 0, sizeof(*C));
  C->cappl = 64;
  C->pl = (plane_t*)xrealloc(NULL, sizeof(plane_t) * C->cappl);
  C->capv = 128;
  C->v = (vert_t*)xrealloc(NULL, sizeof(vert_t) * C->capv);
  C->out = (int*)xrealloc(NULL, sizeof(int) * C->capv);
  C->removed = (int*)xrealloc(NULL, sizeof(int) * C->capv);
  C->caplist = 256;
  C->list = (int*)xrealloc(NULL, sizeof(int) * C->caplist);
  C->capvtmp = 128;
  C->vtmp = (vert_t*)xrealloc(NULL, sizeof(vert_t) * C->capvtmp);
}

static void cell_free_storage(cell_t* C) {
  free(C->pl);
  free(C->v);
  free(C->out);
  free(C->removed);
  free(C->list);
  free(C->vtmp);
}

static void ensure_vcap(cell_t* C, int need) {
  if (need <= C->capv) return;
  while (C->capv < need) C->capv *= 2;
  C->v = (vert_t*)xrealloc(C->v, sizeof(vert_t) * C->capv);
  C->out = (int*)xrealloc(C->out, sizeof(int) * C->capv);
  C->removed = (int*)xrealloc(C->removed, sizeof(int) * C->capv);
}

static int add_plane(cell_t* C, const plane_t* P) {
  if (C->npl == C->cappl) {
    C->cappl *= 2;
    C->pl = (plane_t*)xrealloc(C->pl, sizeof(plane_t) * C->cappl);
  }
  C->pl[C->npl] = *P;
  return C->npl++;
}

/* site plane of j for cell i, local coordinates around p_i */
static void make_site_plane(const problem_t* pr, int64_t i, int64_t j, plane_t* P) {
  double wi = site_w(pr, i);
  double wj = site_w(pr, j);
  double nn = 0.0;
  for (int k = 0; k < 3; k++) {
    P->n[k] = site_x(pr, j, k) - site_x(pr, i, k);
    nn += P->n[k] * P->n[k];
  }
  P->b = 0.5 * (nn + (wi - wj));
  P->bmag = 0.5 * (nn + fabs(wi) + fabs(wj));
  P->site = j;
  P->owner = i;
  if (pr->exact) {
    int64_t nn_i = 0;
    for (int k = 0; k < 3; k++) {
      int64_t d = pr->X[3 * j + k] - pr->X[3 * i + k];
      P->N[k] = 2 * d;
      nn_i += d * d;
    }
    P->B = nn_i + (pr->W[i] - pr->W[j]);
  }
}

/* box face k: 0:+x 1:-x 2:+y 3:-y 4:+z 5:-z */
static void make_box_plane(const problem_t* pr, int64_t i, int k, plane_t* P) {
  int ax = k >> 1;
  double s = (k & 1) ? -1.0 : 1.0;
  double pi = site_x(pr, i, ax);
  P->n[0] = P->n[1] = P->n[2] = 0.0;
  P->n[ax] = s;
  P->b = (k & 1) ? (pi - pr->lo[ax]) : (pr->hi[ax] - pi);
  P->bmag = fabs(P->b);
  P->site = -1 - k;
  P->owner = i;
  if (pr->exact) {
    P->N[0] = P->N[1] = P->N[2] = 0;
    P->N[ax] = (k & 1) ? -1 : 1;
    P->B = (k & 1) ? (pr->X[3 * i + ax] - pr->LO[ax]) : (pr->HI[ax] - pr->X[3 * i + ax]);
  }
}

static double det3(const double r0[3], const double r1[3], const double r2[3]) {
  return r0[0] * (r1[1] * r2[2] - r1[2] * r2[1]) - r0[1] * (r1[0] * r2[2] - r1[2] * r2[0]) +
         r0[2] * (r1[0] * r2[1] - r1[1] * r2[0]);
}

static double perm3(const double r0[3], const double r1[3], const double r2[3]) {
  return r0[0] * (r1[1] * r2[2] + r1[2] * r2[1]) + r0[1] * (r1[0] * r2[2] + r1[2] * r2[0]) +
         r0[2] * (r1[0] * r2[1] + r1[1] * r2[0]);
}

static i128 det3i(const i128 r0[3], const i128 r1[3], const i128 r2[3]) {
  return r0[0] * (r1[1] * r2[2] - r1[2] * r2[1]) - r0[1] * (r1[0] * r2[2] - r1[2] * r2[0]) +
         r0[2] * (r1[0] * r2[1] - r1[1] * r2[0]);
}

/* Fill the Cramer numerators/denominator, permanents, position and its
 * error bound of vertex (a,b,c). */
static void vertex_from_planes(const cell_t* C, int exact, int a, int b, int c, vert_t* V) {
  const plane_t* P[3] = {&C->pl[a], &C->pl[b], &C->pl[c]};
  V->p[0] = a;
  V->p[1] = b;
  V->p[2] = c;
  double N[3][3], M[3][3];
  for (int r = 0; r < 3; r++)
    for (int k = 0; k < 3; k++) {
      N[r][k] = P[r]->n[k];
      M[r][k] = fabs(P[r]->n[k]);
    }
  /* D0 */
  V->D[3] = det3(N[0], N[1], N[2]);
  V->P[3] = perm3(M[0], M[1], M[2]);
  /* Dk: column k replaced by b */
  for (int k = 0; k < 3; k++) {
    double R[3][3], RM[3][3];
    for (int r = 0; r < 3; r++) {
      for (int q = 0; q < 3; q++) {
        R[r][q] = N[r][q];
        RM[r][q] = M[r][q];
      }
      R[r][k] = P[r]->b;
      RM[r][k] = P[r]->bmag;
    }
    V->D[k] = det3(R[0], R[1], R[2]);
    V->P[k] = perm3(RM[0], RM[1], RM[2]);
  }
  /* position and a bound on its error: each numerator / denominator is
   * within 32*EPS of its permanent (entry rounding of at most 4 EPS
   * relative times 3 factors, plus the cofactor arithmetic) */
  double e0 = 32.0 * EPS * V->P[3];
  double xn = 0.0, en = 0.0;
  for (int k = 0; k < 3; k++) {
    V->x[k] = V->D[k] / V->D[3];
    xn += V->x[k] * V->x[k];
    double ek = 32.0 * EPS * V->P[k];
    en += ek * ek;
  }
  xn = sqrt(xn);
  if (!(fabs(V->D[3]) > 2.0 * e0)) {
    V->err = INFINITY;
  } else {
    V->err = (sqrt(en) + xn * e0) / (fabs(V->D[3]) - e0) * (1.0 + 1e-9) + 4.0 * EPS * xn;
  }
  if (exact) {
    i128 NI[3][3];
    for (int r = 0; r < 3; r++)
      for (int k = 0; k < 3; k++) NI[r][k] = (i128)P[r]->N[k];
    V->E[3] = det3i(NI[0], NI[1], NI[2]);
    for (int k = 0; k < 3; k++) {
      i128 R[3][3];
      for (int r = 0; r < 3; r++) {
        for (int q = 0; q < 3; q++) R[r][q] = NI[r][q];
        R[r][k] = (i128)P[r]->B;
      }
      V->E[k] = det3i(R[0], R[1], R[2]);
    }
  }
}

/* ------------------------------------------------------------------ */
/* exact signs by floating-point expansions (Shewchuk, "Adaptive precision
 * floating-point arithmetic and fast robust geometric predicates", 1997).
 * An expansion is an array of doubles whose exact sum is the value; built
 * only by Grow-Expansion with zero elimination, it is nonoverlapping and
 * ordered by increasing magnitude (Shewchuk's Theorem 10, round-to-nearest),
 * so its sign is the sign of its last component. Inputs here are float32
 * coordinates and weights (or FP64 for a finite-difference override), far
 * from overflow and underflow, so TwoSum and TwoProduct are exact.        */

typedef struct {
  double* c;
  int n, cap;
  int overflow;
} xp_t;

#define XP_CAP 2048

/* a + b = *s + *e exactly (Knuth's TwoSum) */
static void two_sum(double a, double b, double* s, double* e) {
  double x = a + b;
  double bv = x - a;
  double av = x - bv;
  *s = x;
  *e = (a - av) + (b - bv);
}

/* a * b = *p + *e exactly (TwoProduct with a fused multiply-add) */
static void two_prod(double a, double b, double* p, double* e) {
  double x = a * b;
  *p = x;
  *e = fma(a, b, -x);
}

static void xp_init(xp_t* X, double* buf) {
  X->c = buf;
  X->n = 0;
  X->cap = XP_CAP;
  X->overflow = 0;
}

/* X += b (Grow-Expansion, zero components dropped) */
static void xp_grow(xp_t* X, double b) {
  if (b == 0.0) return;
  double q = b;
  int m = 0;
  for (int k = 0; k < X->n; k++) {
    double s, e;
    two_sum(q, X->c[k], &s, &e);
    q = s;
    if (e != 0.0) X->c[m++] = e;
  }
  if (q != 0.0) {
    if (m >= X->cap) {
      X->overflow = 1;
      return;
    }
    X->c[m++] = q;
  }
  X->n = m;
}

static int xp_sign(const xp_t* X) {
  if (X->n == 0) return 0;
  return X->c[X->n - 1] > 0.0 ? 1 : -1;
}

/* X += s * A * B, s = +1 or -1 (every partial product grown in exactly) */
static void xp_add_product(xp_t* X, const xp_t* A, const xp_t* B, double s) {
  for (int a = 0; a < A->n; a++)
    for (int b = 0; b < B->n; b++) {
      double p, e;
      two_prod(A->c[a], B->c[b], &p, &e);
      xp_grow(X, s * e);
      xp_grow(X, s * p);
    }
  if (A->overflow || B->overflow) X->overflow = 1;
}

/* exact row (n, 2b) of a plane, recomputed from the sites: n = p_j - p_i,
 * 2b = |n|^2 + w_i - w_j for site planes, n = +-e_k and 2b = 2 (bound - p)
 * for box faces (doubling 2b for every plane scales T by 2, not its sign) */
typedef struct {
  double nb[3][2], bb[XP_CAP];
  xp_t N[3], B;
} xrow_t;

static void exact_row(const problem_t* pr, const plane_t* P, xrow_t* R) {
  for (int k = 0; k < 3; k++) xp_init(&R->N[k], R->nb[k]);
  xp_init(&R->B, R->bb);
  int64_t i = P->owner;
  if (P->site >= 0) {
    int64_t j = P->site;
    for (int k = 0; k < 3; k++) {
      xp_grow(&R->N[k], site_x(pr, j, k));
      xp_grow(&R->N[k], -site_x(pr, i, k));
      xp_add_product(&R->B, &R->N[k], &R->N[k], 1.0);
    }
    xp_grow(&R->B, site_w(pr, i));
    xp_grow(&R->B, -site_w(pr, j));
  } else {
    int f = (int)(-1 - P->site), ax = f >> 1;
    double sg = (f & 1) ? -1.0 : 1.0;
    xp_grow(&R->N[ax], sg);
    /* 2 (hi - p) or 2 (p - lo): doubling is exact */
    if (f & 1) {
      xp_grow(&R->B, 2.0 * site_x(pr, i, ax));
      xp_grow(&R->B, -2.0 * pr->lo[ax]);
    } else {
      xp_grow(&R->B, 2.0 * pr->hi[ax]);
      xp_grow(&R->B, -2.0 * site_x(pr, i, ax));
    }
  }
}

/* exact 3x3 determinant of rows r0, r1, r2 whose entries are expansions:
 * cofactor expansion along r0, each 2x2 minor formed exactly first */
static void xp_det3(const xp_t* r0[3], const xp_t* r1[3], const xp_t* r2[3], xp_t* D, double* m1) {
  xp_init(D, D->c);
  for (int col = 0; col < 3; col++) {
    int c1 = (col + 1) % 3, c2 = (col + 2) % 3;
    xp_t M;
    xp_init(&M, m1);
    xp_add_product(&M, r1[c1], r2[c2], 1.0);
    xp_add_product(&M, r1[c2], r2[c1], -1.0);
    xp_add_product(D, r0[col], &M, 1.0);
    if (M.overflow) D->overflow = 1;
  }
}

/* exact sign of s_v = n_h . v - b_h for the vertex of planes (a, b, c):
 * sign(T) * sign(D0), with T = n_h . (D1, D2, D3) - b_h D0 and v = D / D0.
 * Returns +1 / -1, 0 when s_v = 0 or D0 = 0, 2 when an expansion ran out
 * of room. */
static int exact_side(const problem_t* pr, const plane_t* Pa, const plane_t* Pb, const plane_t* Pc,
                      const plane_t* Ph) {
  xrow_t* R = (xrow_t*)xrealloc(NULL, sizeof(xrow_t) * 4);
  double* buf = (double*)xrealloc(NULL, sizeof(double) * XP_CAP * 8);
  exact_row(pr, Pa, &R[0]);
  exact_row(pr, Pb, &R[1]);
  exact_row(pr, Pc, &R[2]);
  exact_row(pr, Ph, &R[3]);
  const xp_t* rows[3][3];
  for (int r = 0; r < 3; r++)
    for (int k = 0; k < 3; k++) rows[r][k] = &R[r].N[k];
  xp_t D0, Dk, T;
  xp_init(&D0, buf);
  xp_det3(rows[0], rows[1], rows[2], &D0, buf + 2 * XP_CAP);
  xp_init(&T, buf + 4 * XP_CAP);
  xp_add_product(&T, &R[3].B, &D0, -1.0);
  for (int k = 0; k < 3; k++) {
    const xp_t* rk[3][3];
    for (int r = 0; r < 3; r++)
      for (int q = 0; q < 3; q++) rk[r][q] = q == k ? &R[r].B : &R[r].N[q];
    xp_init(&Dk, buf + 5 * XP_CAP);
    xp_det3(rk[0], rk[1], rk[2], &Dk, buf + 2 * XP_CAP);
    xp_add_product(&T, &R[3].N[k], &Dk, 1.0);
  }
  int over = D0.overflow || T.overflow;
  for (int r = 0; r < 4; r++) over |= R[r].B.overflow;
  int sd = xp_sign(&D0), st = xp_sign(&T);
  free(R);
  free(buf);
  if (over) return 2;
  return sd * st;
}

/* +1: vertex strictly outside plane H, 0: inside or on it. */
static int vertex_outside(const problem_t* pr, const cell_t* C, const vert_t* V, const plane_t* H, int64_t* stats) {
  if (pr->exact) {
    i128 T = (i128)H->N[0] * V->E[0] + (i128)H->N[1] * V->E[1] + (i128)H->N[2] * V->E[2] -
             (i128)H->B * V->E[3];
    if (T == 0) stats[ST_DEGENERATE]++;
    return T > 0;
  }
  double T = H->n[0] * V->D[0] + H->n[1] * V->D[1] + H->n[2] * V->D[2] - H->b * V->D[3];
  double bound = 64.0 * EPS *
                 (fabs(H->n[0]) * V->P[0] + fabs(H->n[1]) * V->P[1] + fabs(H->n[2]) * V->P[2] +
                  H->bmag * V->P[3]);
  if (fabs(T) > bound) return T > 0.0;
  stats[ST_EXACT]++;
  int sg = exact_side(pr, &C->pl[V->p[0]], &C->pl[V->p[1]], &C->pl[V->p[2]], H);
  if (sg == 2) { /* could not certify: keep the FP64 sign and say so */
    stats[ST_AMBIGUOUS]++;
    return T > 0.0;
  }
  if (sg == 0) stats[ST_DEGENERATE]++;
  return sg > 0;
}

/* start the cell as the box (App. B "Initialization", with the user box) */
static void cell_start(const problem_t* pr, int64_t i, cell_t* C) {
  C->npl = 0;
  C->nv = 0;
  C->empty = 0;
  for (int k = 0; k < 6; k++) {
    plane_t P;
    make_box_plane(pr, i, k, &P);
    add_plane(C, &P);
  }
  ensure_vcap(C, 8);
  for (int sx = 0; sx < 2; sx++)
    for (int sy = 0; sy < 2; sy++)
      for (int sz = 0; sz < 2; sz++) {
        int a = 0 + sx, b = 2 + sy, c = 4 + sz;
        int neg = (sx + sy + sz) & 1; /* det(±e_x, ±e_y, ±e_z) < 0 */
        if (neg) {
          int t = b;
          b = c;
          c = t;
        }
        vertex_from_planes(C, pr->exact, a, b, c, &C->v[C->nv++]);
      }
}

/* does vertex V contain the cyclic ordered pair (u,v)? */
static int has_pair(const vert_t* V, int u, int v) {
  return (V->p[0] == u && V->p[1] == v) || (V->p[1] == u && V->p[2] == v) ||
         (V->p[2] == u && V->p[0] == v);
}

/* third plane of V given that it contains the cyclic pair (u,v) */
static int third_of(const vert_t* V, int u, int v) {
  for (int k = 0; k < 3; k++)
    if (V->p[k] != u && V->p[k] != v) return V->p[k];
  return -1;
}

/* Clip by one half-space (App. B "Clipping by a half-space").
 * Returns 0 on success. */
static int cell_clip(const problem_t* pr, cell_t* C, const plane_t* H, int64_t* stats) {
  stats[ST_TESTS]++;
  int nv = C->nv, nout = 0;
  /* step 1: classify every vertex */
  for (int k = 0; k < nv; k++) {
    C->out[k] = vertex_outside(pr, C, &C->v[k], H, stats);
    C->removed[k] = 0;
    nout += C->out[k];
  }
  if (nout == 0) return 0; /* plane misses the cell */
  stats[ST_CLIPS]++;
  if (nout == nv) { /* everything removed: empty cell */
    C->empty = 1;
    C->nv = 0;
    return 0;
  }
  /* step 2: remove marked vertices one at a time, each adjacent to the
   * current hole, keeping the hole boundary as a circular plane list */
  int first = -1;
  for (int k = 0; k < nv; k++)
    if (C->out[k]) {
      first = k;
      break;
    }
  int* L = C->list;
  int m = 3;
  L[0] = C->v[first].p[0];
  L[1] = C->v[first].p[1];
  L[2] = C->v[first].p[2];
  C->removed[first] = 1;
  int nrem = 1;
  while (nrem < nout) {
    int progressed = 0;
    for (int t = 0; t < m && !progressed; t++) {
      int a = L[t], b = L[(t + 1) % m];
      /* the kept-or-not vertex across dangling edge (a,b) holds pair (b,a) */
      int k;
      for (k = 0; k < nv; k++)
        if (!C->removed[k] && has_pair(&C->v[k], b, a)) break;
      if (k == nv || !C->out[k]) continue;
      int x = third_of(&C->v[k], b, a);
      /* local update: (a,b) becomes (a,x),(x,b) */
      if (m + 1 >= C->caplist) {
        C->caplist *= 2;
        C->list = L = (int*)xrealloc(C->list, sizeof(int) * C->caplist);
      }
      for (int q = m; q > t + 1; q--) L[q] = L[q - 1];
      L[t + 1] = x;
      m++;
      C->removed[k] = 1;
      nrem++;
      progressed = 1;
      /* an edge of the removed vertex already on the boundary appears
       * twice in a row as (u,v),(v,u): both become interior */
      int changed = 1;
      while (changed && m > 3) {
        changed = 0;
        for (int q = 0; q < m; q++) {
          if (L[q] == L[(q + 2) % m]) {
            int r1 = (q + 1) % m, r2 = (q + 2) % m;
            int lo_i = r1 < r2 ? r1 : r2, hi_i = r1 < r2 ? r2 : r1;
            for (int s = hi_i; s < m - 1; s++) L[s] = L[s + 1];
            m--;
            for (int s = lo_i; s < m - 1; s++) L[s] = L[s + 1];
            m--;
            changed = 1;
            break;
          }
        }
      }
    }
    if (!progressed) {
      stats[ST_TOPO_FAIL]++;
      return ORC_ERR_TOPOLOGY;
    }
  }
  /* every boundary pair must now lead to a kept vertex */
  for (int t = 0; t < m; t++) {
    int a = L[t], b = L[(t + 1) % m];
    int k;
    for (k = 0; k < nv; k++)
      if (!C->removed[k] && has_pair(&C->v[k], b, a)) break;
    if (k == nv || C->out[k]) {
      stats[ST_TOPO_FAIL]++;
      return ORC_ERR_TOPOLOGY;
    }
  }
  /* step 3: append the new half-space and close the hole */
  int h = add_plane(C, H);
  int nkeep = nv - nout;
  int nnew = nkeep + m;
  if (nnew > C->capvtmp) {
    while (C->capvtmp < nnew) C->capvtmp *= 2;
    C->vtmp = (vert_t*)xrealloc(C->vtmp, sizeof(vert_t) * C->capvtmp);
  }
  int q = 0;
  for (int k = 0; k < nv; k++)
    if (!C->out[k]) C->vtmp[q++] = C->v[k];
  for (int t = 0; t < m; t++) {
    vert_t* V = &C->vtmp[q++];
    vertex_from_planes(C, pr->exact, L[t], L[(t + 1) % m], h, V);
    if (pr->exact && V->E[3] <= 0) stats[ST_ORIENT_FAIL]++;
  }
  ensure_vcap(C, nnew);
  memcpy(C->v, C->vtmp, sizeof(vert_t) * nnew);
  C->nv = nnew;
  return 0;
}

/* isotropic security radius: upper bound of max_v |v~| */
static double cell_radius(const cell_t* C) {
  double R = 0.0;
  for (int k = 0; k < C->nv; k++) {
    const vert_t* V = &C->v[k];
    double r = sqrt(V->x[0] * V->x[0] + V->x[1] * V->x[1] + V->x[2] * V->x[2]) + V->err;
    R = dmax(R, r);
  }
  return R * (1.0 + 1e-12);
}

/* ------------------------------------------------------------------ */
/* duplicate positions (d_ij undefined): larger weight wins, then lower
 * index; the loser's cell is empty                                      */

static int is_duplicate(const problem_t* pr, int64_t i, int64_t j) {
  return pr->xyz[3 * i] == pr->xyz[3 * j] && pr->xyz[3 * i + 1] == pr->xyz[3 * j + 1] &&
         pr->xyz[3 * i + 2] == pr->xyz[3 * j + 2];
}

static int duplicate_beats(const problem_t* pr, int64_t i, int64_t j) {
  double wi = pr->w ? pr->w[i] : 0.0, wj = pr->w ? pr->w[j] : 0.0;
  return (wj > wi) || (wj == wi && j < i);
}

/* power distance from p_i to the plane of j (Eq. 2) */
static double plane_distance(const problem_t* pr, int64_t i, int64_t j) {
  double D2 = 0.0;
  for (int k = 0; k < 3; k++) {
    double d = (double)pr->xyz[3 * j + k] - (double)pr->xyz[3 * i + k];
    D2 += d * d;
  }
  double wi = pr->w ? pr->w[i] : 0.0, wj = pr->w ? pr->w[j] : 0.0;
  if (D2 == 0.0) return -INFINITY;
  return (D2 + wi - wj) / (2.0 * sqrt(D2));
}

/* ------------------------------------------------------------------ */
/* k-d tree with per-node maximum weight                                */

typedef struct {
  double lo[3], hi[3];
  double wmax;
  int64_t left, right; /* -1 for leaves */
  int64_t start, count;
} kdnode_t;

typedef struct {
  kdnode_t* nodes;
  int64_t nnodes, cap;
  int64_t* idx;
  int64_t root;
} kdtree_t;

static float coord_of(const problem_t* pr, int64_t i, int ax) { return pr->xyz[3 * i + ax]; }

static void kd_select(const problem_t* pr, int64_t* a, int64_t n, int64_t kth, int ax) {
  /* quickselect on coordinate ax; ties broken by index for determinism */
  int64_t lo = 0, hi = n - 1;
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    float pv = coord_of(pr, a[mid], ax);
    int64_t piv = a[mid];
    int64_t i = lo, j = hi;
    while (i <= j) {
      while (coord_of(pr, a[i], ax) < pv || (coord_of(pr, a[i], ax) == pv && a[i] < piv)) i++;
      while (coord_of(pr, a[j], ax) > pv || (coord_of(pr, a[j], ax) == pv && a[j] > piv)) j--;
      if (i <= j) {
        int64_t t = a[i];
        a[i] = a[j];
        a[j] = t;
        i++;
        j--;
      }
    }
    if (kth <= j)
      hi = j;
    else if (kth >= i)
      lo = i;
    else
      return;
  }
}

static int64_t kd_build_rec(kdtree_t* T, const problem_t* pr, int64_t start, int64_t count) {
  if (T->nnodes == T->cap) {
    T->cap *= 2;
    T->nodes = (kdnode_t*)xrealloc(T->nodes, sizeof(kdnode_t) * T->cap);
  }
  int64_t id = T->nnodes++;
  kdnode_t nd;
  for (int k = 0; k < 3; k++) {
    nd.lo[k] = INFINITY;
    nd.hi[k] = -INFINITY;
  }
  nd.wmax = -INFINITY;
  for (int64_t q = start; q < start + count; q++) {
    int64_t s = T->idx[q];
    for (int k = 0; k < 3; k++) {
      double c = pr->xyz[3 * s + k];
      if (c < nd.lo[k]) nd.lo[k] = c;
      if (c > nd.hi[k]) nd.hi[k] = c;
    }
    double ws = pr->w ? pr->w[s] : 0.0;
    if (ws > nd.wmax) nd.wmax = ws;
  }
  nd.start = start;
  nd.count = count;
  nd.left = nd.right = -1;
  if (count > 8) {
    int ax = 0;
    for (int k = 1; k < 3; k++)
      if (nd.hi[k] - nd.lo[k] > nd.hi[ax] - nd.lo[ax]) ax = k;
    int64_t half = count / 2;
    kd_select(pr, T->idx + start, count, half, ax);
    int64_t l = kd_build_rec(T, pr, start, half);
    int64_t r = kd_build_rec(T, pr, start + half, count - half);
    nd.left = l;
    nd.right = r;
  }
  T->nodes[id] = nd;
  return id;
}

static void kd_build(kdtree_t* T, const problem_t* pr) {
  T->cap = 1024;
  T->nnodes = 0;
  T->nodes = (kdnode_t*)xrealloc(NULL, sizeof(kdnode_t) * T->cap);
  T->idx = (int64_t*)xrealloc(NULL, sizeof(int64_t) * (size_t)pr->n);
  for (int64_t q = 0; q < pr->n; q++) T->idx[q] = q;
  T->root = kd_build_rec(T, pr, 0, pr->n);
}

static void kd_free(kdtree_t* T) {
  free(T->nodes);
  free(T->idx);
}

/* Lower bound of d_ij over all sites of a node (Sec. 4.2.2). A site j of
 * the node lies at distance D in [dmin, dmax] from p_i (nearest and
 * farthest point of the node's box) and has w_j <= wmax, so
 *   d_ij = D/2 + (w_i - w_j)/(2D) >= f(D) = D/2 + c/(2D),  c = w_i - wmax.
 * For c <= 0, f increases with D and the bound is f(dmin) (the paper's);
 * for c > 0, f is convex with its minimum at D = sqrt(c), so the bound is
 * f at sqrt(c) clamped to [dmin, dmax]. */
static double node_lower_bound(const problem_t* pr, int64_t i, const kdnode_t* nd) {
  double d2 = 0.0, f2 = 0.0;
  for (int k = 0; k < 3; k++) {
    double c = pr->xyz[3 * i + k];
    double e = 0.0;
    if (c < nd->lo[k]) e = nd->lo[k] - c;
    if (c > nd->hi[k]) e = c - nd->hi[k];
    d2 += e * e;
    double f = dmax(fabs(c - nd->lo[k]), fabs(nd->hi[k] - c));
    f2 += f * f;
  }
  double wi = pr->w ? pr->w[i] : 0.0;
  double c = wi - nd->wmax;
  double D = sqrt(d2);
  if (c > 0.0) {
    double s = sqrt(c), dm = sqrt(f2);
    D = s < D ? D : (s > dm ? dm : s);
  }
  if (D == 0.0) return -INFINITY;
  return 0.5 * D + c / (2.0 * D);
}

/* binary min-heap of (key, kind, id) */
typedef struct {
  double key;
  int64_t id; /* >= 0: node id; < 0: site -1-j */
} hitem_t;

typedef struct {
  hitem_t* a;
  int64_t n, cap;
} heap_t;

static void heap_push(heap_t* H, double key, int64_t id) {
  if (H->n == H->cap) {
    H->cap = H->cap ? 2 * H->cap : 256;
    H->a = (hitem_t*)xrealloc(H->a, sizeof(hitem_t) * H->cap);
  }
  int64_t k = H->n++;
  while (k > 0) {
    int64_t p = (k - 1) / 2;
    if (H->a[p].key < key || (H->a[p].key == key && H->a[p].id <= id)) break;
    H->a[k] = H->a[p];
    k = p;
  }
  H->a[k].key = key;
  H->a[k].id = id;
}

static hitem_t heap_pop(heap_t* H) {
  hitem_t top = H->a[0];
  hitem_t last = H->a[--H->n];
  int64_t k = 0;
  for (;;) {
    int64_t c = 2 * k + 1;
    if (c >= H->n) break;
    if (c + 1 < H->n &&
        (H->a[c + 1].key < H->a[c].key || (H->a[c + 1].key == H->a[c].key && H->a[c + 1].id < H->a[c].id)))
      c++;
    if (last.key < H->a[c].key || (last.key == H->a[c].key && last.id <= H->a[c].id)) break;
    H->a[k] = H->a[c];
    k = c;
  }
  H->a[k] = last;
  return top;
}

/* ------------------------------------------------------------------ */
/* one cell                                                             */

typedef struct {
  int64_t* cand; /* brute mode: candidate indices */
  double* keys;
  heap_t heap;
} qscratch_t;

/* sort candidates by (key, index) */
static void sort_candidates(int64_t* idx, double* key, int64_t n, int64_t* tmpi, double* tmpk) {
  /* bottom-up merge sort, stable, keyed by (key, idx) */
  for (int64_t width = 1; width < n; width *= 2) {
    for (int64_t lo = 0; lo < n; lo += 2 * width) {
      int64_t mid = lo + width < n ? lo + width : n;
      int64_t hi = lo + 2 * width < n ? lo + 2 * width : n;
      int64_t a = lo, b = mid, o = lo;
      while (a < mid && b < hi) {
        if (key[a] < key[b] || (key[a] == key[b] && idx[a] < idx[b])) {
          tmpi[o] = idx[a];
          tmpk[o++] = key[a++];
        } else {
          tmpi[o] = idx[b];
          tmpk[o++] = key[b++];
        }
      }
      while (a < mid) {
        tmpi[o] = idx[a];
        tmpk[o++] = key[a++];
      }
      while (b < hi) {
        tmpi[o] = idx[b];
        tmpk[o++] = key[b++];
      }
    }
    memcpy(idx, tmpi, sizeof(int64_t) * n);
    memcpy(key, tmpk, sizeof(double) * n);
  }
}

/* process candidate j for cell i; returns <0 on error, 1 if the cell
 * became empty */
static int offer_candidate(const problem_t* pr, int64_t i, int64_t j, cell_t* C, int64_t* stats) {
  if (pr->dup_loser[j]) return 0; /* implied by its duplicate's plane */
  if (is_duplicate(pr, i, j)) {
    if (duplicate_beats(pr, i, j)) {
      C->empty = 1;
      C->nv = 0;
      return 1;
    }
    return 0;
  }
  plane_t P;
  make_site_plane(pr, i, j, &P);
  int rc = cell_clip(pr, C, &P, stats);
  if (rc < 0) return rc;
  return C->empty ? 1 : 0;
}

static int build_cell(const problem_t* pr, const kdtree_t* T, int mode, int64_t i, cell_t* C,
                      qscratch_t* S, int64_t* stats) {
  cell_start(pr, i, C);
  if (pr->dup_loser[i]) { /* an exact duplicate site beats this one */
    C->empty = 1;
    C->nv = 0;
    stats[ST_EMPTY]++;
    return 0;
  }
  if (mode == 0) {
    /* brute force: every other site, ascending d_ij */
    int64_t m = 0;
    for (int64_t j = 0; j < pr->n; j++) {
      if (j == i) continue;
      S->cand[m] = j;
      S->keys[m] = plane_distance(pr, i, j);
      m++;
    }
    sort_candidates(S->cand, S->keys, m, S->cand + pr->n, S->keys + pr->n);
    for (int64_t q = 0; q < m; q++) {
      int rc = offer_candidate(pr, i, S->cand[q], C, stats);
      if (rc < 0) return rc;
      if (rc == 1) break;
    }
  } else {
    /* k-d tree stream in ascending lower bound of d_ij */
    heap_t* H = &S->heap;
    H->n = 0;
    heap_push(H, node_lower_bound(pr, i, &T->nodes[T->root]), T->root);
    double R = cell_radius(C);
    while (H->n > 0) {
      hitem_t it = heap_pop(H);
      if (it.key > R) break; /* nothing left can reach the cell */
      if (it.id >= 0) {
        const kdnode_t* nd = &T->nodes[it.id];
        if (nd->left < 0) {
          for (int64_t q = nd->start; q < nd->start + nd->count; q++) {
            int64_t j = T->idx[q];
            if (j == i) continue;
            heap_push(H, plane_distance(pr, i, j), -1 - j);
          }
        } else {
          heap_push(H, node_lower_bound(pr, i, &T->nodes[nd->left]), nd->left);
          heap_push(H, node_lower_bound(pr, i, &T->nodes[nd->right]), nd->right);
        }
      } else {
        int64_t j = -1 - it.id;
        int rc = offer_candidate(pr, i, j, C, stats);
        if (rc < 0) return rc;
        if (rc == 1) break;
        R = cell_radius(C);
      }
    }
  }
  if (C->empty) stats[ST_EMPTY]++;
  return 0;
}

/* ------------------------------------------------------------------ */
/* faces, volume, centroid, neighbours                                  */

/* Successor of vertex v = (f,p,q) on face f is the vertex holding the
 * cyclic pair (f,q): the other end of edge f∩q. Walking successors gives
 * the face polygon counter-clockwise about the outward normal. */
static int rot_to(const vert_t* V, int f, int* p, int* q) {
  for (int k = 0; k < 3; k++)
    if (V->p[k] == f) {
      *p = V->p[(k + 1) % 3];
      *q = V->p[(k + 2) % 3];
      return 1;
    }
  return 0;
}

/* gather face f's polygon in order; returns its length or -1 */
static int face_polygon(const cell_t* C, int f, int* poly, int cap) {
  int start = -1, cnt = 0;
  for (int k = 0; k < C->nv; k++) {
    int p, q;
    if (rot_to(&C->v[k], f, &p, &q)) {
      if (start < 0) start = k;
      cnt++;
    }
  }
  if (start < 0) return 0;
  if (cnt > cap) return -1;
  int len = 0, cur = start;
  do {
    if (len >= cnt) return -1;
    poly[len++] = cur;
    int p = -1, q = -1;
    rot_to(&C->v[cur], f, &p, &q);
    int nxt = -1;
    for (int k = 0; k < C->nv; k++)
      if (k != cur && has_pair(&C->v[k], f, q)) {
        nxt = k;
        break;
      }
    if (nxt < 0) return -1;
    cur = nxt;
  } while (cur != start);
  return len == cnt ? len : -1;
}

static void cross3(const double a[3], const double b[3], double r[3]) {
  r[0] = a[1] * b[2] - a[2] * b[1];
  r[1] = a[2] * b[0] - a[0] * b[2];
  r[2] = a[0] * b[1] - a[1] * b[0];
}

/* volume and first moment (about the local origin p_i) by tetrahedra
 * (c, x0, xk, xk+1) over every fan-triangulated face */
static int cell_volume(const cell_t* C, double* vol, double mom[3], int* poly, int cap, int64_t* stats) {
  double c[3] = {0, 0, 0};
  for (int k = 0; k < C->nv; k++)
    for (int a = 0; a < 3; a++) c[a] += C->v[k].x[a];
  for (int a = 0; a < 3; a++) c[a] /= (double)C->nv;
  double V = 0.0, M[3] = {0, 0, 0};
  for (int f = 0; f < C->npl; f++) {
    int len = face_polygon(C, f, poly, cap);
    if (len < 0) {
      stats[ST_FACEWALK_FAIL]++;
      return ORC_ERR_TOPOLOGY;
    }
    if (len < 3) continue;
    const double* x0 = C->v[poly[0]].x;
    for (int t = 1; t + 1 < len; t++) {
      const double* x1 = C->v[poly[t]].x;
      const double* x2 = C->v[poly[t + 1]].x;
      double a0[3], a1[3], a2[3], cr[3];
      for (int a = 0; a < 3; a++) {
        a0[a] = x0[a] - c[a];
        a1[a] = x1[a] - c[a];
        a2[a] = x2[a] - c[a];
      }
      cross3(a1, a2, cr);
      double tv = (a0[0] * cr[0] + a0[1] * cr[1] + a0[2] * cr[2]) / 6.0;
      V += tv;
      for (int a = 0; a < 3; a++) M[a] += tv * (a0[a] + a1[a] + a2[a]) / 4.0;
    }
  }
  *vol = V;
  for (int a = 0; a < 3; a++) mom[a] = M[a] + V * c[a];
  return 0;
}

/* ------------------------------------------------------------------ */
/* public entry points                                                  */

static const problem_t* g_cmp_pr;

static int cmp_position(const void* A, const void* B) {
  int64_t a = *(const int64_t*)A, b = *(const int64_t*)B;
  const float* x = g_cmp_pr->xyz;
  for (int k = 0; k < 3; k++) {
    if (x[3 * a + k] < x[3 * b + k]) return -1;
    if (x[3 * a + k] > x[3 * b + k]) return 1;
  }
  return a < b ? -1 : (a > b);
}

static void mark_duplicate_losers(problem_t* pr) {
  int64_t n = pr->n;
  pr->dup_loser = (unsigned char*)xrealloc(NULL, (size_t)n);
  memset(pr->dup_loser, 0, (size_t)n);
  int64_t* idx = (int64_t*)xrealloc(NULL, sizeof(int64_t) * (size_t)n);
  for (int64_t q = 0; q < n; q++) idx[q] = q;
  g_cmp_pr = pr;
  qsort(idx, (size_t)n, sizeof(int64_t), cmp_position);
  for (int64_t a = 0; a < n;) {
    int64_t b = a + 1;
    while (b < n && pr->xyz[3 * idx[b]] == pr->xyz[3 * idx[a]] && pr->xyz[3 * idx[b] + 1] == pr->xyz[3 * idx[a] + 1] &&
           pr->xyz[3 * idx[b] + 2] == pr->xyz[3 * idx[a] + 2])
      b++;
    for (int64_t u = a; u < b; u++)
      for (int64_t v = a; v < b; v++)
        if (u != v && duplicate_beats(pr, idx[u], idx[v])) pr->dup_loser[idx[u]] = 1;
    a = b;
  }
  free(idx);
}

static void free_problem(problem_t* pr) {
  free(pr->X);
  free(pr->W);
  free(pr->dup_loser);
}

static int setup_problem(problem_t* pr, const float* xyz, const float* w, int64_t n, const float* lo,
                         const float* hi, int exact) {
  memset(pr, 0, sizeof(*pr));
  pr->ov_site = -1;
  pr->xyz = xyz;
  pr->w = w;
  pr->n = n;
  pr->exact = exact;
  for (int k = 0; k < 3; k++) {
    pr->lo[k] = lo[k];
    pr->hi[k] = hi[k];
    if (!(pr->lo[k] < pr->hi[k])) return ORC_ERR_ARG;
  }
  for (int64_t q = 0; q < 3 * n; q++)
    if (!isfinite(xyz[q])) return ORC_ERR_ARG;
  if (w)
    for (int64_t q = 0; q < n; q++)
      if (!isfinite(w[q])) return ORC_ERR_ARG;
  if (exact) {
    const double SX = 1048576.0;            /* 2^20 */
    const double SW = 1099511627776.0;      /* 2^40 */
    pr->X = (int64_t*)xrealloc(NULL, sizeof(int64_t) * 3 * (size_t)n);
    pr->W = (int64_t*)xrealloc(NULL, sizeof(int64_t) * (size_t)n);
    for (int64_t q = 0; q < 3 * n; q++) {
      double s = (double)xyz[q] * SX;
      if (s != floor(s) || fabs(s) > 4.0 * SX) return ORC_ERR_GRID;
      pr->X[q] = (int64_t)s;
    }
    for (int64_t q = 0; q < n; q++) {
      double s = w ? (double)w[q] * SW : 0.0;
      if (s != floor(s) || fabs(s) > 4.0 * SW) return ORC_ERR_GRID;
      pr->W[q] = (int64_t)s;
    }
    for (int k = 0; k < 3; k++) {
      double a = pr->lo[k] * SX, b = pr->hi[k] * SX;
      if (a != floor(a) || b != floor(b) || fabs(a) > 4.0 * SX || fabs(b) > 4.0 * SX) return ORC_ERR_GRID;
      pr->LO[k] = (int64_t)a;
      pr->HI[k] = (int64_t)b;
    }
  }
  mark_duplicate_losers(pr);
  return 0;
}



/*
 * oracle_cells: neighbours, volume and centroid of the requested cells.
 *   xyz [3n] float32 sites, w [n] float32 weights or NULL, lo/hi [3] box.
 *   cells [ncells] int64 site indices (NULL: all n, in order).
 *   mode 0 = brute force, 1 = k-d tree. exact 1 = integer predicates.
 *   counts [ncells] int32, offsets [ncells+1] int64 and nbrs [nbr_cap] int32
 *   (CSR, ascending within a row; if the total exceeds nbr_cap nothing is
 *   written to nbrs and stats[ST_N] receives the required size),
 *   vol [ncells], cen [3*ncells] float64, nverts / nfaces [ncells] int32
 *   (may be NULL), stats [ST_N] int64 (summed over cells).
 * Returns 0 or a negative error code. stats has ST_N + 1 entries.
 */
typedef struct {
  int32_t* v;
  int64_t n, cap;
} ibuf_t;

static void ibuf_push(ibuf_t* b, int32_t x) {
  if (b->n == b->cap) {
    b->cap = b->cap ? 2 * b->cap : 4096;
    b->v = (int32_t*)xrealloc(b->v, sizeof(int32_t) * (size_t)b->cap);
  }
  b->v[b->n++] = x;
}

/* the cells of one problem whose set-up (and k-d tree, mode 1) is done */
static int cells_run(const problem_t* prp, const kdtree_t* Tp, int mode, const int64_t* cells, int64_t ncells,
                     int32_t* counts, int64_t* offsets, int32_t* nbrs, int64_t nbr_cap, double* vol, double* cen,
                     int32_t* nverts, int32_t* nfaces, int64_t* stats, int nthreads) {
  const problem_t pr = *prp;
  const kdtree_t T = *Tp;
  const float* xyz = pr.xyz;
  const int64_t n = pr.n;
  if (!cells) ncells = n;
  for (int k = 0; k <= ST_N; k++) stats[k] = 0;
  int err = 0;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
  int nth = omp_get_max_threads();
#else
  (void)nthreads;
  int nth = 1;
#endif
  /* per-thread neighbour lists, copied out in cell order afterwards */
  ibuf_t* tb = (ibuf_t*)calloc((size_t)nth, sizeof(ibuf_t));
  int64_t* where = (int64_t*)xrealloc(NULL, sizeof(int64_t) * (size_t)(ncells > 0 ? ncells : 1));
  int* owner = (int*)xrealloc(NULL, sizeof(int) * (size_t)(ncells > 0 ? ncells : 1));
#pragma omp parallel
  {
#ifdef _OPENMP
    int tid = omp_get_thread_num();
#else
    int tid = 0;
#endif
    ibuf_t* mybuf = &tb[tid];
    cell_t C;
    cell_init_storage(&C);
    qscratch_t S;
    memset(&S, 0, sizeof(S));
    if (mode == 0) {
      S.cand = (int64_t*)xrealloc(NULL, sizeof(int64_t) * 2 * (size_t)n);
      S.keys = (double*)xrealloc(NULL, sizeof(double) * 2 * (size_t)n);
    }
    int polycap = 4096;
    int* poly = (int*)xrealloc(NULL, sizeof(int) * polycap);
    int nbcap = 4096;
    int* nb = (int*)xrealloc(NULL, sizeof(int) * (size_t)nbcap);
    int64_t* tmpn = (int64_t*)xrealloc(NULL, sizeof(int64_t) * (size_t)nbcap);
    int64_t st[ST_N];
    for (int k = 0; k < ST_N; k++) st[k] = 0;
#pragma omp for schedule(dynamic, 8)
    for (int64_t q = 0; q < ncells; q++) {
      int64_t i = cells ? cells[q] : q;
      if (i < 0 || i >= n) {
#pragma omp atomic write
        err = ORC_ERR_ARG;
        continue;
      }
      int r = build_cell(&pr, &T, mode, i, &C, &S, st);
      if (r < 0) {
#pragma omp atomic write
        err = r;
        continue;
      }
      double p[3] = {xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2]};
      where[q] = 0;
      owner[q] = tid;
      if (C.empty || C.nv == 0) {
        counts[q] = 0;
        vol[q] = 0.0;
        for (int a = 0; a < 3; a++) cen[3 * q + a] = p[a];
        if (nverts) nverts[q] = 0;
        if (nfaces) nfaces[q] = 0;
        continue;
      }
      /* neighbours: site planes referenced by a final vertex */
      if (C.npl > nbcap) {
        nbcap = 2 * C.npl;
        nb = (int*)xrealloc(nb, sizeof(int) * (size_t)nbcap);
        tmpn = (int64_t*)xrealloc(tmpn, sizeof(int64_t) * (size_t)nbcap);
      }
      for (int f = 0; f < C.npl; f++) nb[f] = 0;
      for (int k = 0; k < C.nv; k++)
        for (int a = 0; a < 3; a++) nb[C.v[k].p[a]] = 1;
      int cnt = 0, nf = 0;
      for (int f = 0; f < C.npl; f++)
        if (nb[f]) {
          nf++;
          if (C.pl[f].site >= 0) tmpn[cnt++] = C.pl[f].site;
        }
      /* ascending */
      for (int a = 1; a < cnt; a++) {
        int64_t x = tmpn[a];
        int b = a - 1;
        while (b >= 0 && tmpn[b] > x) {
          tmpn[b + 1] = tmpn[b];
          b--;
        }
        tmpn[b + 1] = x;
      }
      counts[q] = cnt;
      where[q] = mybuf->n;
      for (int a = 0; a < cnt; a++) ibuf_push(mybuf, (int32_t)tmpn[a]);
      if (nverts) nverts[q] = C.nv;
      if (nfaces) nfaces[q] = nf;
      double V, M[3];
      if (C.nv > polycap) {
        polycap = C.nv * 2;
        poly = (int*)xrealloc(poly, sizeof(int) * polycap);
      }
      r = cell_volume(&C, &V, M, poly, polycap, st);
      if (r < 0) {
#pragma omp atomic write
        err = r;
        continue;
      }
      vol[q] = V;
      for (int a = 0; a < 3; a++) cen[3 * q + a] = p[a] + M[a] / V;
    }
#pragma omp critical
    {
      for (int k = 0; k < ST_N; k++) stats[k] += st[k];
    }
    cell_free_storage(&C);
    free(S.cand);
    free(S.keys);
    free(S.heap.a);
    free(poly);
    free(nb);
    free(tmpn);
  }
  offsets[0] = 0;
  for (int64_t q = 0; q < ncells; q++) offsets[q + 1] = offsets[q] + (err ? 0 : counts[q]);
  stats[ST_N] = offsets[ncells];
  if (!err && nbrs && offsets[ncells] <= nbr_cap) {
    for (int64_t q = 0; q < ncells; q++)
      if (counts[q] > 0) memcpy(nbrs + offsets[q], tb[owner[q]].v + where[q], sizeof(int32_t) * (size_t)counts[q]);
  } else if (!err && offsets[ncells] > nbr_cap) {
    err = ORC_ERR_NBR_CAP;
  }
  for (int t = 0; t < nth; t++) free(tb[t].v);
  free(tb);
  free(where);
  free(owner);
  return err;
}

int oracle_cells(const float* xyz, const float* w, int64_t n, const float* lo, const float* hi,
                 const int64_t* cells, int64_t ncells, int mode, int exact, int32_t* counts,
                 int64_t* offsets, int32_t* nbrs, int64_t nbr_cap, double* vol, double* cen, int32_t* nverts,
                 int32_t* nfaces, int64_t* stats, int nthreads) {
  if (n <= 0 || !xyz || !lo || !hi || !counts || !offsets || !vol || !cen || !stats) return ORC_ERR_ARG;
  problem_t pr;
  int rc = setup_problem(&pr, xyz, w, n, lo, hi, exact);
  if (rc) {
    free_problem(&pr);
    return rc;
  }
  kdtree_t T;
  memset(&T, 0, sizeof(T));
  if (mode == 1) kd_build(&T, &pr);
  rc = cells_run(&pr, &T, mode, cells, ncells, counts, offsets, nbrs, nbr_cap, vol, cen, nverts, nfaces, stats,
                 nthreads);
  if (mode == 1) kd_free(&T);
  free_problem(&pr);
  return rc;
}

/*
 * A session keeps one problem's set-up (duplicate marks, k-d tree) between
 * calls, so that many samples of cells of one large point set do not each
 * rebuild the tree. The caller's xyz / w arrays must outlive the session.
 * oracle_session_cells takes the arguments of oracle_cells from `cells` on.
 */
typedef struct {
  problem_t pr;
  kdtree_t T;
  int mode;
} session_t;

void* oracle_session_open(const float* xyz, const float* w, int64_t n, const float* lo, const float* hi, int mode,
                          int exact, int* rc) {
  *rc = ORC_ERR_ARG;
  if (n <= 0 || !xyz || !lo || !hi) return NULL;
  session_t* S = (session_t*)calloc(1, sizeof(session_t));
  if (!S) {
    *rc = ORC_ERR_MEM;
    return NULL;
  }
  *rc = setup_problem(&S->pr, xyz, w, n, lo, hi, exact);
  if (*rc) {
    free_problem(&S->pr);
    free(S);
    return NULL;
  }
  S->mode = mode;
  if (mode == 1) kd_build(&S->T, &S->pr);
  return S;
}

int oracle_session_cells(void* h, const int64_t* cells, int64_t ncells, int32_t* counts, int64_t* offsets,
                         int32_t* nbrs, int64_t nbr_cap, double* vol, double* cen, int32_t* nverts, int32_t* nfaces,
                         int64_t* stats, int nthreads) {
  session_t* S = (session_t*)h;
  if (!S || !counts || !offsets || !vol || !cen || !stats) return ORC_ERR_ARG;
  return cells_run(&S->pr, &S->T, S->mode, cells, ncells, counts, offsets, nbrs, nbr_cap, vol, cen, nverts, nfaces,
                   stats, nthreads);
}

void oracle_session_close(void* h) {
  session_t* S = (session_t*)h;
  if (!S) return;
  if (S->mode == 1) kd_free(&S->T);
  free_problem(&S->pr);
  free(S);
}

/*
 * oracle_grad: gradient of L = sum_i c_i V_i + d_i . g_i (g = centroid)
 * with respect to site positions and weights, accumulated over the cells
 * listed in `cells` (NULL: all). With all cells listed, gp/gw are the full
 * gradient; with a subset, gp[k]/gw[k] are exact for any site k whose own
 * cell and every neighbour cell are in the subset.
 *
 * Reynolds transport with fixed combinatorics: on face F_ij of cell i
 * (area A, unit outward normal (p_j-p_i)/D) the boundary moves with normal
 * speed (p_j - x).dp_j / D, (x - p_i).dp_i / D, dw_i / 2D and -dw_j / 2D
 * (differentiate |x-p_i|^2 - w_i - |x-p_j|^2 + w_j = 0 and divide by its
 * gradient 2D). Hence, with x~ = x - p_i and over F_ij:
 *   dV/dp_j = int (n - x~) dA / D      dV/dp_i = int x~ dA / D
 *   dV/dw_i = A / 2D                   dV/dw_j = -A / 2D
 *   dM~/dp_j = int x~ (n - x~)^T dA/D  dM~/dp_i = int x~ x~^T dA / D
 *   dM~/dw_i = int x~ dA / 2D          dM~/dw_j = -int x~ dA / 2D
 * where M~ = int x~ dV, and dg = (dM~ - g~ dV) / V with g~ = g - p_i.
 * Box faces do not move. Face integrals use fan triangles with
 *   int_T x x^T dA = A_T/12 (sum_k v_k v_k^T + s s^T),  s = sum_k v_k.
 * cvec [n], dvec [3n] float64; gp [3n], gw [n] float64 accumulated (+=).
 */
int oracle_grad(const float* xyz, const float* w, int64_t n, const float* lo, const float* hi,
                const int64_t* cells, int64_t ncells, const double* cvec, const double* dvec,
                double* gp, double* gw, int64_t* stats, int nthreads) {
  if (n <= 0 || !xyz || !cvec || !dvec || !gp || !gw || !stats) return ORC_ERR_ARG;
  problem_t pr;
  int rc = setup_problem(&pr, xyz, w, n, lo, hi, 0);
  if (rc) {
    free_problem(&pr);
    return rc;
  }
  if (!cells) ncells = n;
  kdtree_t T;
  kd_build(&T, &pr);
  for (int k = 0; k < ST_N; k++) stats[k] = 0;
  int err = 0;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
#pragma omp parallel
  {
    cell_t C;
    cell_init_storage(&C);
    qscratch_t S;
    memset(&S, 0, sizeof(S));
    int polycap = 4096;
    int* poly = (int*)xrealloc(NULL, sizeof(int) * polycap);
    int64_t st[ST_N];
    for (int k = 0; k < ST_N; k++) st[k] = 0;
#pragma omp for schedule(dynamic, 8)
    for (int64_t q = 0; q < ncells; q++) {
      int64_t i = cells ? cells[q] : q;
      int r = build_cell(&pr, &T, 1, i, &C, &S, st);
      if (r < 0) {
#pragma omp atomic write
        err = r;
        continue;
      }
      if (C.empty || C.nv == 0) continue;
      double V, M[3];
      if (C.nv > polycap) {
        polycap = 2 * C.nv;
        poly = (int*)xrealloc(poly, sizeof(int) * polycap);
      }
      r = cell_volume(&C, &V, M, poly, polycap, st);
      if (r < 0) {
#pragma omp atomic write
        err = r;
        continue;
      }
      double g[3] = {M[0] / V, M[1] / V, M[2] / V}; /* local centroid g~ */
      double ci = cvec[i];
      const double* di = &dvec[3 * i];
      double gpi[3] = {0, 0, 0}, gwi = 0.0;
      for (int f = 0; f < C.npl; f++) {
        const plane_t* P = &C.pl[f];
        if (P->site < 0) continue;
        int len = face_polygon(&C, f, poly, polycap);
        if (len < 3) continue;
        double D = sqrt(P->n[0] * P->n[0] + P->n[1] * P->n[1] + P->n[2] * P->n[2]);
        double u[3] = {P->n[0] / D, P->n[1] / D, P->n[2] / D};
        double A = 0.0, Am[3] = {0, 0, 0}, S2[3][3] = {{0}};
        const double* x0 = C.v[poly[0]].x;
        for (int t = 1; t + 1 < len; t++) {
          const double* x1 = C.v[poly[t]].x;
          const double* x2 = C.v[poly[t + 1]].x;
          double e1[3], e2[3], cr[3];
          for (int a = 0; a < 3; a++) {
            e1[a] = x1[a] - x0[a];
            e2[a] = x2[a] - x0[a];
          }
          cross3(e1, e2, cr);
          double at = 0.5 * (cr[0] * u[0] + cr[1] * u[1] + cr[2] * u[2]);
          double s[3];
          for (int a = 0; a < 3; a++) s[a] = x0[a] + x1[a] + x2[a];
          A += at;
          for (int a = 0; a < 3; a++) Am[a] += at * s[a] / 3.0;
          for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++)
              S2[a][b] += at / 12.0 * (x0[a] * x0[b] + x1[a] * x1[b] + x2[a] * x2[b] + s[a] * s[b]);
        }
        int64_t j = P->site;
        /* dV and dM~ for the four parameter groups, chained into L */
        double dVdpj[3], dVdpi[3], dMdpj[3][3], dMdpi[3][3];
        for (int a = 0; a < 3; a++) {
          dVdpj[a] = (A * P->n[a] - Am[a]) / D;
          dVdpi[a] = Am[a] / D;
          for (int b = 0; b < 3; b++) {
            dMdpj[a][b] = (Am[a] * P->n[b] - S2[a][b]) / D; /* d M~_a / d p_j,b */
            dMdpi[a][b] = S2[a][b] / D;
          }
        }
        double dVdwi = A / (2.0 * D), dVdwj = -A / (2.0 * D);
        double dMdwi[3], dMdwj[3];
        for (int a = 0; a < 3; a++) {
          dMdwi[a] = Am[a] / (2.0 * D);
          dMdwj[a] = -Am[a] / (2.0 * D);
        }
        /* dL = c dV + d . (dM~ - g~ dV) / V */
        double gj[3], gi[3];
        for (int b = 0; b < 3; b++) {
          double sj = ci * dVdpj[b], si = ci * dVdpi[b];
          for (int a = 0; a < 3; a++) {
            sj += di[a] * (dMdpj[a][b] - g[a] * dVdpj[b]) / V;
            si += di[a] * (dMdpi[a][b] - g[a] * dVdpi[b]) / V;
          }
          gj[b] = sj;
          gi[b] = si;
        }
        double wj_ = ci * dVdwj, wi_ = ci * dVdwi;
        for (int a = 0; a < 3; a++) {
          wj_ += di[a] * (dMdwj[a] - g[a] * dVdwj) / V;
          wi_ += di[a] * (dMdwi[a] - g[a] * dVdwi) / V;
        }
        for (int b = 0; b < 3; b++) {
#pragma omp atomic
          gp[3 * j + b] += gj[b];
          gpi[b] += gi[b];
        }
#pragma omp atomic
        gw[j] += wj_;
        gwi += wi_;
      }
      for (int b = 0; b < 3; b++) {
#pragma omp atomic
        gp[3 * i + b] += gpi[b];
      }
#pragma omp atomic
      gw[i] += gwi;
    }
#pragma omp critical
    {
      for (int k = 0; k < ST_N; k++) stats[k] += st[k];
    }
    cell_free_storage(&C);
    free(S.heap.a);
    free(poly);
  }
  kd_free(&T);
  free_problem(&pr);
  return err;
}

/*
 * oracle_certify: for every final vertex v of each listed cell i and every
 * site m != i, check pow(v, i) <= pow(v, m) (v lies inside the half-space of
 * m; with the exact predicate this is the empty-sphere test of the dual
 * regular triangulation). out_viol [ncells] int64 receives the number of
 * violating (vertex, site) pairs per cell; stats as in oracle_cells.
 */
int oracle_certify(const float* xyz, const float* w, int64_t n, const float* lo, const float* hi,
                   const int64_t* cells, int64_t ncells, int exact, int64_t* out_viol, int64_t* stats,
                   int nthreads) {
  if (n <= 0 || !xyz || !out_viol || !stats) return ORC_ERR_ARG;
  problem_t pr;
  int rc = setup_problem(&pr, xyz, w, n, lo, hi, exact);
  if (rc) {
    free_problem(&pr);
    return rc;
  }
  if (!cells) ncells = n;
  kdtree_t T;
  kd_build(&T, &pr);
  for (int k = 0; k < ST_N; k++) stats[k] = 0;
  int err = 0;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
#pragma omp parallel
  {
    cell_t C;
    cell_init_storage(&C);
    qscratch_t S;
    memset(&S, 0, sizeof(S));
    int64_t st[ST_N];
    for (int k = 0; k < ST_N; k++) st[k] = 0;
#pragma omp for schedule(dynamic, 4)
    for (int64_t q = 0; q < ncells; q++) {
      int64_t i = cells ? cells[q] : q;
      out_viol[q] = 0;
      int r = build_cell(&pr, &T, 1, i, &C, &S, st);
      if (r < 0) {
#pragma omp atomic write
        err = r;
        continue;
      }
      for (int k = 0; k < C.nv; k++)
        for (int64_t mm = 0; mm < n; mm++) {
          if (mm == i || is_duplicate(&pr, i, mm)) continue;
          /* the vertex lies on its own defining planes by construction */
          if (C.pl[C.v[k].p[0]].site == mm || C.pl[C.v[k].p[1]].site == mm ||
              C.pl[C.v[k].p[2]].site == mm)
            continue;
          plane_t P;
          make_site_plane(&pr, i, mm, &P);
          if (vertex_outside(&pr, &C, &C.v[k], &P, st)) out_viol[q]++;
        }
    }
#pragma omp critical
    {
      for (int k = 0; k < ST_N; k++) stats[k] += st[k];
    }
    cell_free_storage(&C);
    free(S.heap.a);
  }
  kd_free(&T);
  free_problem(&pr);
  return err;
}

/* the oracle's own vertices of one cell: positions [3*cap] and plane
 * triplets mapped to sites (-1-k for box faces) [3*cap]; returns the
 * vertex count, or a negative error */
int oracle_cell_vertices(const float* xyz, const float* w, int64_t n, const float* lo, const float* hi,
                         int64_t i, int mode, int exact, double* pos, int64_t* tri, int32_t cap) {
  problem_t pr;
  int rc = setup_problem(&pr, xyz, w, n, lo, hi, exact);
  if (rc) {
    free_problem(&pr);
    return rc;
  }
  kdtree_t T;
  memset(&T, 0, sizeof(T));
  if (mode == 1) kd_build(&T, &pr);
  cell_t C;
  cell_init_storage(&C);
  qscratch_t S;
  memset(&S, 0, sizeof(S));
  if (mode == 0) {
    S.cand = (int64_t*)xrealloc(NULL, sizeof(int64_t) * 2 * (size_t)n);
    S.keys = (double*)xrealloc(NULL, sizeof(double) * 2 * (size_t)n);
  }
  int64_t st[ST_N] = {0};
  int r = build_cell(&pr, &T, mode, i, &C, &S, st);
  int out = r;
  if (r == 0) {
    out = C.nv;
    if (C.nv > cap) out = ORC_ERR_NBR_CAP;
    else
      for (int k = 0; k < C.nv; k++)
        for (int a = 0; a < 3; a++) {
          pos[3 * k + a] = C.v[k].x[a];
          tri[3 * k + a] = C.pl[C.v[k].p[a]].site;
        }
  }
  cell_free_storage(&C);
  free(S.cand);
  free(S.keys);
  free(S.heap.a);
  if (mode == 1) kd_free(&T);
  free_problem(&pr);
  return out;
}

/* Cell i as the box clipped by the planes of its neighbour row only (the
 * combinatorics held fixed); its volume and first moment about p_i. */
static int fd_cell(const problem_t* pr, int64_t i, const int64_t* offsets, const int32_t* nbrs, cell_t* C,
                   int* poly, int cap, int64_t* stats, double* V, double mom[3]) {
  cell_start(pr, i, C);
  for (int64_t e = offsets[i]; e < offsets[i + 1] && !C->empty; e++) {
    plane_t P;
    make_site_plane(pr, i, (int64_t)nbrs[e], &P);
    int r = cell_clip(pr, C, &P, stats);
    if (r < 0) return r;
  }
  *V = 0.0;
  mom[0] = mom[1] = mom[2] = 0.0;
  if (C->empty || C->nv == 0) return 0;
  return cell_volume(C, V, mom, poly, cap, stats);
}

/*
 * oracle_fd_grad: central finite differences of L = sum_i c_i V_i + d_i . g_i
 * (V_i volume, g_i centroid) with respect to the coordinates and the weight
 * of each listed site, with the cell combinatorics held fixed as in the
 * analytic gradient: moving site k moves only faces of cell k and of its
 * neighbours' cells, so L changes only through those cells; each is rebuilt,
 * with site k moved in FP64, as the box clipped by the planes of its own
 * neighbour row of the unperturbed diagram. A cell with an empty row is an
 * empty cell and contributes nothing (its gradient is 0 by the convention of
 * the analytic gradient, although its reported centroid is its site).
 *   offsets [n+1] int64, nbrs int32: the diagram's CSR over all n sites.
 *   c [n], d [3n] float64: the loss coefficients.
 *   sites [m] int64; hx [m] position steps, hw [m] weight steps (absolute;
 *   hw unused without weights).
 *   gp [3m] and gw [m] (NULL without weights) float64 out.
 * Returns 0 or a negative error code.
 */
int oracle_fd_grad(const float* xyz, const float* w, int64_t n, const float* lo, const float* hi,
                   const int64_t* offsets, const int32_t* nbrs, const double* c, const double* d,
                   const int64_t* sites, int64_t m, const double* hx, const double* hw, double* gp, double* gw,
                   int nthreads) {
  if (n <= 0 || !xyz || !offsets || !nbrs || !c || !d || !sites || !hx || !gp || (w && (!hw || !gw)))
    return ORC_ERR_ARG;
  problem_t base;
  int rc = setup_problem(&base, xyz, w, n, lo, hi, 0);
  if (rc) {
    free_problem(&base);
    return rc;
  }
  int err = 0;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
#pragma omp parallel
  {
    problem_t pr = base;
    cell_t C;
    cell_init_storage(&C);
    int cap = 4096;
    int* poly = (int*)xrealloc(NULL, sizeof(int) * cap);
    int64_t st[ST_N];
    for (int k = 0; k < ST_N; k++) st[k] = 0;
#pragma omp for schedule(dynamic, 4)
    for (int64_t q = 0; q < m; q++) {
      const int64_t k = sites[q];
      if (k < 0 || k >= n) {
#pragma omp atomic write
        err = ORC_ERR_ARG;
        continue;
      }
      const int nparam = w ? 4 : 3;
      for (int a = 0; a < nparam; a++) {
        const double h = a < 3 ? hx[q] : hw[q];
        double Ls[2] = {0.0, 0.0};
        for (int s = 0; s < 2; s++) {
          pr.ov_site = k;
          for (int t = 0; t < 3; t++) pr.ov_xyz[t] = (double)xyz[3 * k + t];
          pr.ov_w = w ? (double)w[k] : 0.0;
          if (a < 3)
            pr.ov_xyz[a] += s ? -h : h;
          else
            pr.ov_w += s ? -h : h;
          double L = 0.0;
          for (int64_t e = offsets[k] - 1; e < offsets[k + 1]; e++) {
            const int64_t i = e < offsets[k] ? k : (int64_t)nbrs[e];
            if (offsets[i + 1] == offsets[i]) continue; /* an empty cell: gradient 0 by convention */
            double V, mom[3];
            int r = fd_cell(&pr, i, offsets, nbrs, &C, poly, cap, st, &V, mom);
            if (r < 0) {
#pragma omp atomic write
              err = r;
              break;
            }
            double g[3];
            for (int t = 0; t < 3; t++) g[t] = site_x(&pr, i, t) + (V > 0.0 ? mom[t] / V : 0.0);
            L += c[i] * V + d[3 * i] * g[0] + d[3 * i + 1] * g[1] + d[3 * i + 2] * g[2];
          }
          Ls[s] = L;
        }
        const double g = (Ls[0] - Ls[1]) / (2.0 * h);
        if (a < 3)
          gp[3 * q + a] = g;
        else
          gw[q] = g;
      }
    }
    free(poly);
    cell_free_storage(&C);
  }
  free_problem(&base);
  return err;
}

/*
 * oracle_exact_side: the exact sign, from the expansion arithmetic above, of
 * s_v = n_h . v - b_h where v is the vertex of the planes of ids[0..2] in the
 * frame of site i and h the plane of ids[3] (ids: site index, or -1-f for
 * box face f). Returns +1, -1, 0 (s_v = 0 or the three planes are
 * dependent), 2 (no room), or ORC_ERR_ARG. A testing entry point.
 */
int oracle_exact_side(const float* xyz, const float* w, int64_t n, const float* lo, const float* hi, int64_t i,
                      const int64_t* ids) {
  if (n <= 0 || !xyz || !lo || !hi || !ids || i < 0 || i >= n) return ORC_ERR_ARG;
  problem_t pr;
  memset(&pr, 0, sizeof(pr));
  pr.ov_site = -1;
  pr.xyz = xyz;
  pr.w = w;
  pr.n = n;
  for (int k = 0; k < 3; k++) {
    pr.lo[k] = lo[k];
    pr.hi[k] = hi[k];
  }
  plane_t P[4];
  for (int k = 0; k < 4; k++) {
    if (ids[k] >= n || ids[k] < -6 || ids[k] == i) return ORC_ERR_ARG;
    if (ids[k] >= 0)
      make_site_plane(&pr, i, ids[k], &P[k]);
    else
      make_box_plane(&pr, i, (int)(-1 - ids[k]), &P[k]);
  }
  return exact_side(&pr, &P[0], &P[1], &P[2], &P[3]);
}

int oracle_stat_count(void) { return ST_N; }
