/*
 * mg_oracle.c -- plain FP64 CPU oracle for the leading-order squared matrix
 * element |M|^2, summed over helicities and colours, per event.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
 * legs of bench.py load this library.  It shares no code, header, table or
 * constant generator with the CUDA path, and the CUDA path never calls it.
 *
 * What is computed (paper Sect. 1: the matrix element of a Monte Carlo event
 * generator, computed per event from Feynman diagrams and helicity
 * amplitudes; Sect. 3: its double-precision reference):
 *
 *   ME = (1/IDEN) * sum_{spin states} sum_{colours} |M|^2
 *
 * with IDEN = initial spin x colour average x final identical-particle
 * factor.  The oracle evaluates the same quantity by an independent exact
 * method:
 *
 *   - e+ e- -> mu+ mu-: the two s-channel diagrams (photon, Z) written out
 *     with explicit 4x4 Dirac matrices;
 *   - u u~ -> t t~: the s-channel gluon diagram with explicit Dirac matrices
 *     and an explicit sum over every colour index;
 *   - u u~ -> t t~ g g: colour-dressed Berends-Giele recursion over both
 *     quark lines with explicit T^a and f^{abc}, every colour summed (the
 *     same recursion reproduces the u u~ -> t t~ and u u~ -> t t~ g results
 *     of the independent evaluations);
 *   - g g -> t t~ + (n-2) g: colour decomposition on one quark line,
 *       M = sum_{sigma in S_n} (T^{a_sigma1} ... T^{a_sigman})_{i_t j_tbar} A(sigma),
 *     partial amplitudes A(sigma) from colour-ordered Berends-Giele recursion
 *     (the alternative to diagrams that the paper cites in Sect. 1), and the
 *     colour sum  sum_col |M|^2 = sum_{sigma,tau} A(sigma)^* C(sigma,tau) A(tau)
 *     with C built from explicit index sums over Gell-Mann matrices.
 *
 * Feynman rules (Peskin & Schroeder conventions, D = d - i g_s T^a A^a):
 *   quark-gluon vertex  i g gamma^mu T^a
 *   three-gluon vertex  g f^{abc} [g^{mu nu}(k-p)^rho + g^{nu rho}(p-q)^mu + g^{rho mu}(q-k)^nu]
 *   four-gluon vertex   -i g^2 [f^{abe}f^{cde}(g^{mu rho}g^{nu sigma} - g^{mu sigma}g^{nu rho}) + ...]
 *   gluon propagator    -i g_{mu nu} / P^2          (Feynman gauge)
 *   top propagator      i (P-slash + m) / (P^2 - m^2 + i m Gamma)   (every top propagator)
 * Substituting f^{abc} T^c = -i [T^a, T^b] gives the colour-ordered current
 *   J(1..m) = (1/P^2) [ -g sum_k V3(J(1..k), J(k+1..m))
 *                       + g^2 sum_{k<l} (2 (J_L.J_R) J_M - (J_L.J_M) J_R - (J_M.J_R) J_L) ]
 *   V3(a,b) = (J_a.J_b)(k_a-k_b) + J_b (2k_b+k_a).J_a - J_a (2k_a+k_b).J_b
 * (all gluon momenta incoming).  External states: Dirac-representation
 * spinors in the spin-z basis (Bjorken-Drell normalisation, ubar u = 2m) and
 * real linear gluon polarisations with eps^0 = 0, eps.k = 0 in the lab frame.
 * Any complete basis gives the same spin sum.
 *
 * Pins (tests/): closed-form e+e- -> mu+mu- (photon and photon+Z), the
 * analytic g g -> t t~ result, Ward identities of every partial amplitude,
 * Bose symmetry, Lorentz invariance, spinor/polarisation completeness,
 * Gell-Mann algebra identities and a colour-dressed recursion with explicit
 * f^{abc} summed over every colour assignment.
 */
#include <complex.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <tgmath.h>

/* Arithmetic type: double by default; the same source built with
 * -DORACLE_REAL="long double" gives the extended-precision variant used to
 * adjudicate disagreements at the 1e-12 level. */
#ifndef ORACLE_REAL
#define ORACLE_REAL double
#endif
typedef ORACLE_REAL real;
typedef ORACLE_REAL complex cplx;
static const real PI_R = 3.14159265358979323846264338327950288L;

#define MGO_OK 0
#define MGO_ERR_ARG (-1)
#define MGO_ERR_NOMEM (-2)

enum {
  MGO_EEMUMU = 0,
  MGO_GGTT = 1,
  MGO_GGTTG = 2,
  MGO_GGTTGG = 3,
  MGO_GGTTGGG = 4,
  MGO_UUTT = 5,
  MGO_UUTTG = 6,
  MGO_UUTTGG = 7
};

#define MAXG 5     /* at most 5 gluons */
#define MAXPERM 120

typedef struct {
  real mt, wt, alpha_s, mz, wz, alpha_em_inv, gf;
  int photon_only;
} oparams;

static void unpack_params(const double* p, oparams* o) {
  o->mt = p[0];
  o->wt = p[1];
  o->alpha_s = p[2];
  o->mz = p[3];
  o->wz = p[4];
  o->alpha_em_inv = p[5];
  o->gf = p[6];
  o->photon_only = (p[7] != 0.0);
}

/* ------------------------------------------------------------------ */
/* Lorentz and Dirac algebra, Dirac representation                    */
/* ------------------------------------------------------------------ */

static cplx GAM[4][4][4]; /* GAM[mu] = gamma^mu                   */
static cplx GAM5[4][4];   /* gamma^5 = i g0 g1 g2 g3               */
static cplx TGEN[8][3][3]; /* T^a = lambda^a / 2                   */

static void matmul4(const cplx a[4][4], const cplx b[4][4], cplx c[4][4]) {
  for (int i = 0; i < 4; i++)
    for (int j = 0; j < 4; j++) {
      cplx s = 0;
      for (int k = 0; k < 4; k++) s += a[i][k] * b[k][j];
      c[i][j] = s;
    }
}

__attribute__((constructor)) static void init_tables(void) {
  memset(GAM, 0, sizeof(GAM));
  /* gamma^0 = diag(1,1,-1,-1); gamma^i = [[0, sigma_i], [-sigma_i, 0]] */
  GAM[0][0][0] = 1; GAM[0][1][1] = 1; GAM[0][2][2] = -1; GAM[0][3][3] = -1;
  const cplx sig[3][2][2] = {{{0, 1}, {1, 0}}, {{0, -I}, {I, 0}}, {{1, 0}, {0, -1}}};
  for (int i = 0; i < 3; i++)
    for (int r = 0; r < 2; r++)
      for (int c = 0; c < 2; c++) {
        GAM[i + 1][r][c + 2] = sig[i][r][c];
        GAM[i + 1][r + 2][c] = -sig[i][r][c];
      }
  cplx t1[4][4], t2[4][4];
  matmul4((const cplx(*)[4])GAM[0], (const cplx(*)[4])GAM[1], t1);
  matmul4((const cplx(*)[4])t1, (const cplx(*)[4])GAM[2], t2);
  matmul4((const cplx(*)[4])t2, (const cplx(*)[4])GAM[3], t1);
  for (int r = 0; r < 4; r++)
    for (int c = 0; c < 4; c++) GAM5[r][c] = I * t1[r][c];

  /* Gell-Mann matrices, T^a = lambda^a / 2 */
  memset(TGEN, 0, sizeof(TGEN));
  TGEN[0][0][1] = 0.5; TGEN[0][1][0] = 0.5;
  TGEN[1][0][1] = -0.5 * I; TGEN[1][1][0] = 0.5 * I;
  TGEN[2][0][0] = 0.5; TGEN[2][1][1] = -0.5;
  TGEN[3][0][2] = 0.5; TGEN[3][2][0] = 0.5;
  TGEN[4][0][2] = -0.5 * I; TGEN[4][2][0] = 0.5 * I;
  TGEN[5][1][2] = 0.5; TGEN[5][2][1] = 0.5;
  TGEN[6][1][2] = -0.5 * I; TGEN[6][2][1] = 0.5 * I;
  const real r3 = 1 / (2 * sqrt((real)3));
  TGEN[7][0][0] = r3; TGEN[7][1][1] = r3; TGEN[7][2][2] = -2.0 * r3;
}

static const real METRIC[4] = {1.0, -1.0, -1.0, -1.0};

static cplx dot_cc(const cplx a[4], const cplx b[4]) {
  return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
}
static cplx dot_rc(const real a[4], const cplx b[4]) {
  return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
}
static real dot_rr(const real a[4], const real b[4]) {
  return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
}

/* S = gamma^mu v_mu for a contravariant complex vector v */
static void slash_c(const cplx v[4], cplx S[4][4]) {
  for (int r = 0; r < 4; r++)
    for (int c = 0; c < 4; c++) {
      cplx s = 0;
      for (int mu = 0; mu < 4; mu++) s += METRIC[mu] * GAM[mu][r][c] * v[mu];
      S[r][c] = s;
    }
}
static void slash_r(const real v[4], cplx S[4][4]) {
  cplx vc[4] = {v[0], v[1], v[2], v[3]};
  slash_c(vc, S);
}

/* row vector times matrix */
static void rowmat(const cplx r[4], const cplx M[4][4], cplx out[4]) {
  for (int c = 0; c < 4; c++) {
    cplx s = 0;
    for (int k = 0; k < 4; k++) s += r[k] * M[k][c];
    out[c] = s;
  }
}
static void matcol(const cplx M[4][4], const cplx v[4], cplx out[4]) {
  for (int r = 0; r < 4; r++) {
    cplx s = 0;
    for (int k = 0; k < 4; k++) s += M[r][k] * v[k];
    out[r] = s;
  }
}
static cplx rowcol(const cplx r[4], const cplx c[4]) {
  cplx s = 0;
  for (int k = 0; k < 4; k++) s += r[k] * c[k];
  return s;
}

/* ------------------------------------------------------------------ */
/* External states                                                    */
/* ------------------------------------------------------------------ */

/* Dirac spinor u(p, s), spin-z basis chi_1 = (1,0), chi_2 = (0,1):
 *   u = [ sqrt(E+m) chi ; (sigma.p) chi / sqrt(E+m) ]                 */
static void spinor_u(const real p[4], real m, int s, cplx u[4]) {
  const real a = sqrt(p[0] + m);
  const cplx chi[2] = {s == 0 ? 1.0 : 0.0, s == 0 ? 0.0 : 1.0};
  /* sigma.p = [[pz, px - i py], [px + i py, -pz]] */
  const cplx sp0 = p[3] * chi[0] + (p[1] - I * p[2]) * chi[1];
  const cplx sp1 = (p[1] + I * p[2]) * chi[0] - p[3] * chi[1];
  u[0] = a * chi[0];
  u[1] = a * chi[1];
  u[2] = sp0 / a;
  u[3] = sp1 / a;
}
/* v(p, s) = [ (sigma.p) eta / sqrt(E+m) ; sqrt(E+m) eta ] */
static void spinor_v(const real p[4], real m, int s, cplx v[4]) {
  const real a = sqrt(p[0] + m);
  const cplx eta[2] = {s == 0 ? 1.0 : 0.0, s == 0 ? 0.0 : 1.0};
  const cplx sp0 = p[3] * eta[0] + (p[1] - I * p[2]) * eta[1];
  const cplx sp1 = (p[1] + I * p[2]) * eta[0] - p[3] * eta[1];
  v[0] = sp0 / a;
  v[1] = sp1 / a;
  v[2] = a * eta[0];
  v[3] = a * eta[1];
}
/* Dirac adjoint psibar = psi^dagger gamma^0 */
static void dirac_bar(const cplx in[4], cplx out[4]) {
  out[0] = conj(in[0]);
  out[1] = conj(in[1]);
  out[2] = -conj(in[2]);
  out[3] = -conj(in[3]);
}

/* Real linear polarisation vectors of a massless vector with momentum k:
 * eps^0 = 0, eps.k = 0, orthonormal.  e1 = unit(n x khat) with n the
 * coordinate axis least aligned with k, e2 = khat x e1.                 */
static void polarisation(const real k[4], int which, real eps[4]) {
  const real kk = sqrt(k[1] * k[1] + k[2] * k[2] + k[3] * k[3]);
  const real kh[3] = {k[1] / kk, k[2] / kk, k[3] / kk};
  int ax = 0;
  for (int i = 1; i < 3; i++)
    if (fabs(kh[i]) < fabs(kh[ax])) ax = i;
  real n[3] = {0, 0, 0};
  n[ax] = 1.0;
  real e1[3] = {n[1] * kh[2] - n[2] * kh[1], n[2] * kh[0] - n[0] * kh[2], n[0] * kh[1] - n[1] * kh[0]};
  const real l1 = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
  for (int i = 0; i < 3; i++) e1[i] /= l1;
  const real e2[3] = {kh[1] * e1[2] - kh[2] * e1[1], kh[2] * e1[0] - kh[0] * e1[2], kh[0] * e1[1] - kh[1] * e1[0]};
  eps[0] = 0.0;
  for (int i = 0; i < 3; i++) eps[i + 1] = (which == 0) ? e1[i] : e2[i];
}

/* ------------------------------------------------------------------ */
/* Permutations (lexicographic order)                                  */
/* ------------------------------------------------------------------ */

static int factorial(int n) {
  int f = 1;
  for (int i = 2; i <= n; i++) f *= i;
  return f;
}

static int next_permutation(int* a, int n) {
  int i = n - 2;
  while (i >= 0 && a[i] >= a[i + 1]) i--;
  if (i < 0) return 0;
  int j = n - 1;
  while (a[j] <= a[i]) j--;
  int t = a[i]; a[i] = a[j]; a[j] = t;
  for (int l = i + 1, r = n - 1; l < r; l++, r--) { t = a[l]; a[l] = a[r]; a[r] = t; }
  return 1;
}

int mgo_permutations(int n, int* perms) {
  if (n < 1 || n > MAXG) return MGO_ERR_ARG;
  int a[MAXG];
  for (int i = 0; i < n; i++) a[i] = i;
  int k = 0;
  do {
    for (int i = 0; i < n; i++) perms[k * n + i] = a[i];
    k++;
  } while (next_permutation(a, n));
  return MGO_OK;
}

/* ------------------------------------------------------------------ */
/* Colour matrix by explicit Gell-Mann index sums                      */
/*   C(sigma,tau) = sum_{a_1..a_n} sum_{i,j}                           */
/*        (T^{a_sigma1}..T^{a_sigman})_{ij} conj((T^{a_tau1}..T^{a_taun})_{ij}) */
/* ------------------------------------------------------------------ */

static void matmul3(const cplx a[3][3], const cplx b[3][3], cplx c[3][3]) {
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) c[i][j] = a[i][0] * b[0][j] + a[i][1] * b[1][j] + a[i][2] * b[2][j];
}

static int colour_matrix_compute(int n, cplx* C) {
  const int np = factorial(n);
  int* perms = (int*)malloc(sizeof(int) * np * n);
  cplx(*W)[3][3] = malloc(sizeof(cplx) * 9 * np);
  if (!perms || !W) { free(perms); free(W); return MGO_ERR_NOMEM; }
  mgo_permutations(n, perms);
  memset(C, 0, sizeof(cplx) * np * np);
  int a[MAXG];
  long total = 1;
  for (int i = 0; i < n; i++) total *= 8;
  for (long code = 0; code < total; code++) {
    long c = code;
    for (int i = 0; i < n; i++) { a[i] = (int)(c % 8); c /= 8; }
    for (int s = 0; s < np; s++) {
      const int* p = perms + s * n;
      cplx acc[3][3], tmp[3][3];
      memcpy(acc, TGEN[a[p[0]]], sizeof(acc));
      for (int l = 1; l < n; l++) {
        matmul3((const cplx(*)[3])acc, (const cplx(*)[3])TGEN[a[p[l]]], tmp);
        memcpy(acc, tmp, sizeof(acc));
      }
      memcpy(W[s], acc, sizeof(acc));
    }
    for (int s = 0; s < np; s++)
      for (int t = s; t < np; t++) {
        cplx sum = 0;
        for (int i = 0; i < 3; i++)
          for (int j = 0; j < 3; j++) sum += W[s][i][j] * conj(W[t][i][j]);
        C[s * np + t] += sum;
      }
  }
  for (int s = 0; s < np; s++)
    for (int t = 0; t < s; t++) C[s * np + t] = conj(C[t * np + s]);
  free(perms);
  free(W);
  return MGO_OK;
}

/* cached per n; computed once under a lock */
static cplx* colour_cache[MAXG + 1];
static pthread_mutex_t colour_lock = PTHREAD_MUTEX_INITIALIZER;

static const cplx* colour_matrix(int n) {
  pthread_mutex_lock(&colour_lock);
  if (!colour_cache[n]) {
    const int np = factorial(n);
    cplx* C = (cplx*)malloc(sizeof(cplx) * np * np);
    if (C && colour_matrix_compute(n, C) == MGO_OK) colour_cache[n] = C;
    else free(C);
  }
  const cplx* r = colour_cache[n];
  pthread_mutex_unlock(&colour_lock);
  return r;
}

int mgo_colour_matrix(int n, double* out /* complex [n!][n!] interleaved */) {
  if (n < 1 || n > MAXG) return MGO_ERR_ARG;
  const cplx* C = colour_matrix(n);
  if (!C) return MGO_ERR_NOMEM;
  const int np = factorial(n);
  for (int i = 0; i < np * np; i++) {
    out[2 * i] = (double)creal(C[i]);
    out[2 * i + 1] = (double)cimag(C[i]);
  }
  return MGO_OK;
}

int mgo_generators(double* out /* complex [8][3][3] */) {
  const cplx* t = &TGEN[0][0][0];
  for (int i = 0; i < 72; i++) {
    out[2 * i] = (double)creal(t[i]);
    out[2 * i + 1] = (double)cimag(t[i]);
  }
  return MGO_OK;
}

/* ------------------------------------------------------------------ */
/* Colour-ordered Berends-Giele recursion                              */
/* ------------------------------------------------------------------ */

typedef struct {
  int n;                      /* number of gluons                         */
  real k[MAXG][4];          /* incoming gluon momenta, by gluon index  */
  cplx eps[MAXG][4];          /* gluon wavefunctions, by gluon index     */
  real pt[4], ptb[4];       /* outgoing top / antitop momenta          */
  cplx ubar[4];               /* Dirac adjoint spinor of the top         */
  cplx v[4];                  /* spinor of the antitop                   */
  real g, mt, wt;
} qline;

/* V3(a,b) = (Ja.Jb)(ka-kb) + Jb (2kb+ka).Ja - Ja (2ka+kb).Jb */
static void vertex3(const real ka[4], const cplx ja[4], const real kb[4], const cplx jb[4], cplx out[4]) {
  real x[4], y[4];
  for (int mu = 0; mu < 4; mu++) {
    x[mu] = 2.0 * kb[mu] + ka[mu];
    y[mu] = 2.0 * ka[mu] + kb[mu];
  }
  const cplx jab = dot_cc(ja, jb);
  const cplx xa = dot_rc(x, ja);
  const cplx yb = dot_rc(y, jb);
  for (int mu = 0; mu < 4; mu++) out[mu] = jab * (ka[mu] - kb[mu]) + jb[mu] * xa - ja[mu] * yb;
}

/* ordered quartic piece: 2(L.R) M - (L.M) R - (M.R) L */
static void vertex4(const cplx l[4], const cplx m[4], const cplx r[4], cplx out[4]) {
  const cplx lr = dot_cc(l, r), lm = dot_cc(l, m), mr = dot_cc(m, r);
  for (int mu = 0; mu < 4; mu++) out[mu] = 2.0 * lr * m[mu] - lm * r[mu] - mr * l[mu];
}

/* Partial amplitude A(sigma) for one ordering sigma of the gluons. */
static cplx ordered_amplitude(const qline* q, const int* sigma) {
  const int n = q->n;
  cplx J[MAXG][MAXG][4];
  real K[MAXG][MAXG][4];
  for (int i = 0; i < n; i++) {
    for (int mu = 0; mu < 4; mu++) {
      J[i][i][mu] = q->eps[sigma[i]][mu];
      K[i][i][mu] = q->k[sigma[i]][mu];
    }
  }
  for (int len = 2; len <= n; len++) {
    for (int i = 0; i + len - 1 < n; i++) {
      const int j = i + len - 1;
      for (int mu = 0; mu < 4; mu++) K[i][j][mu] = K[i][j - 1][mu] + K[j][j][mu];
      cplx acc[4] = {0, 0, 0, 0}, t[4];
      for (int m = i; m < j; m++) {
        vertex3(K[i][m], J[i][m], K[m + 1][j], J[m + 1][j], t);
        for (int mu = 0; mu < 4; mu++) acc[mu] += -q->g * t[mu];
      }
      for (int m1 = i; m1 < j; m1++)
        for (int m2 = m1 + 1; m2 < j; m2++) {
          vertex4(J[i][m1], J[m1 + 1][m2], J[m2 + 1][j], t);
          for (int mu = 0; mu < 4; mu++) acc[mu] += q->g * q->g * t[mu];
        }
      const real p2 = dot_rr(K[i][j], K[i][j]);
      for (int mu = 0; mu < 4; mu++) J[i][j][mu] = acc[mu] / p2;
    }
  }
  /* quark line: Psi[k] = row current with the first k gluons of sigma attached */
  cplx Psi[MAXG][4];
  for (int c = 0; c < 4; c++) Psi[0][c] = q->ubar[c];
  for (int k = 1; k < n; k++) {
    real Q[4];
    for (int mu = 0; mu < 4; mu++) Q[mu] = q->pt[mu] - K[0][k - 1][mu];
    const cplx den = dot_rr(Q, Q) - q->mt * q->mt + I * q->mt * q->wt;
    cplx row[4] = {0, 0, 0, 0}, t[4];
    for (int m = 0; m < k; m++) {
      cplx S[4][4];
      slash_c(J[m][k - 1], S);
      rowmat(Psi[m], (const cplx(*)[4])S, t);
      for (int c = 0; c < 4; c++) row[c] += t[c];
    }
    cplx P[4][4];
    slash_r(Q, P);
    for (int c = 0; c < 4; c++) P[c][c] += q->mt;
    rowmat(row, (const cplx(*)[4])P, t);
    /* (i g) from the vertex, i / den from the propagator */
    for (int c = 0; c < 4; c++) Psi[k][c] = (I * q->g) * (I / den) * t[c];
  }
  cplx amp = 0;
  for (int m = 0; m < n; m++) {
    cplx S[4][4], t[4];
    slash_c(J[m][n - 1], S);
    matcol((const cplx(*)[4])S, q->v, t);
    amp += (I * q->g) * rowcol(Psi[m], t);
  }
  return amp;
}

static void all_ordered_amplitudes(const qline* q, cplx* amps) {
  const int n = q->n;
  int a[MAXG];
  for (int i = 0; i < n; i++) a[i] = i;
  int s = 0;
  do {
    amps[s++] = ordered_amplitude(q, a);
  } while (next_permutation(a, n));
}

static int fill_qline(qline* q, int n, const double* params, const double* kin, const double* eps, const double* pt,
                      const double* ubar, const double* ptb, const double* v) {
  if (n < 1 || n > MAXG) return MGO_ERR_ARG;
  oparams o;
  unpack_params(params, &o);
  q->n = n;
  q->g = sqrt(4.0 * PI_R * o.alpha_s);
  q->mt = o.mt;
  q->wt = o.wt;
  for (int i = 0; i < n; i++)
    for (int mu = 0; mu < 4; mu++) {
      q->k[i][mu] = kin[4 * i + mu];
      q->eps[i][mu] = eps[8 * i + 2 * mu] + I * eps[8 * i + 2 * mu + 1];
    }
  for (int mu = 0; mu < 4; mu++) {
    q->pt[mu] = pt[mu];
    q->ptb[mu] = ptb[mu];
    q->ubar[mu] = ubar[2 * mu] + I * ubar[2 * mu + 1];
    q->v[mu] = v[2 * mu] + I * v[2 * mu + 1];
  }
  return MGO_OK;
}

/* Partial amplitudes for explicit external wavefunctions (test hook):
 * kin = incoming gluon momenta [n][4]; eps complex [n][4]; ubar, v complex [4]. */
int mgo_ordered_amps(int n, const double* params, const double* kin, const double* eps, const double* pt,
                     const double* ubar, const double* ptb, const double* v, double* amps_out) {
  qline q;
  int rc = fill_qline(&q, n, params, kin, eps, pt, ubar, ptb, v);
  if (rc) return rc;
  cplx A[MAXPERM];
  all_ordered_amplitudes(&q, A);
  for (int i = 0; i < factorial(n); i++) {
    amps_out[2 * i] = (double)creal(A[i]);
    amps_out[2 * i + 1] = (double)cimag(A[i]);
  }
  return MGO_OK;
}

/* sum_{sigma,tau} A^*(sigma) C(sigma,tau) A(tau) for explicit external states */
int mgo_ordered_colour_sum(int n, const double* params, const double* kin, const double* eps, const double* pt,
                           const double* ubar, const double* ptb, const double* v, double* out) {
  qline q;
  int rc = fill_qline(&q, n, params, kin, eps, pt, ubar, ptb, v);
  if (rc) return rc;
  const cplx* C = colour_matrix(n);
  if (!C) return MGO_ERR_NOMEM;
  const int np = factorial(n);
  cplx A[MAXPERM];
  all_ordered_amplitudes(&q, A);
  cplx s = 0;
  for (int i = 0; i < np; i++)
    for (int j = 0; j < np; j++) s += conj(A[i]) * C[i * np + j] * A[j];
  *out = creal(s);
  return MGO_OK;
}

/* ------------------------------------------------------------------ */
/* Colour-dressed recursion (pin for the colour decomposition)         */
/* Full Feynman rules with explicit f^{abc} and T^a, currents over     */
/* gluon subsets, summed over every colour assignment of the externals.*/
/* ------------------------------------------------------------------ */

static real FABC[8][8][8];
static int fabc_ready = 0;
static pthread_mutex_t fabc_lock = PTHREAD_MUTEX_INITIALIZER;

/* f^{abc} = -2 i Tr([T^a, T^b] T^c) */
static void init_fabc(void) {
  pthread_mutex_lock(&fabc_lock);
  if (!fabc_ready) {
    for (int a = 0; a < 8; a++)
      for (int b = 0; b < 8; b++)
        for (int c = 0; c < 8; c++) {
          cplx ab[3][3], ba[3][3], x[3][3], y[3][3];
          matmul3((const cplx(*)[3])TGEN[a], (const cplx(*)[3])TGEN[b], ab);
          matmul3((const cplx(*)[3])TGEN[b], (const cplx(*)[3])TGEN[a], ba);
          for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) x[i][j] = ab[i][j] - ba[i][j];
          matmul3((const cplx(*)[3])x, (const cplx(*)[3])TGEN[c], y);
          const cplx tr = y[0][0] + y[1][1] + y[2][2];
          FABC[a][b][c] = creal(-2.0 * I * tr);
        }
    fabc_ready = 1;
  }
  pthread_mutex_unlock(&fabc_lock);
}

int mgo_fabc(double* out /* [8][8][8] */) {
  init_fabc();
  const real* f = &FABC[0][0][0];
  for (int i = 0; i < 512; i++) out[i] = (double)f[i];
  return MGO_OK;
}

typedef struct {
  cplx J[1 << MAXG][8][4]; /* J[subset][colour][mu] */
  real K[1 << MAXG][4];
  int have[1 << MAXG];
} dressed_ws;

static void dressed_current(const qline* q, const int* col, int S, dressed_ws* w) {
  if (w->have[S]) return;
  const int n = q->n;
  for (int mu = 0; mu < 4; mu++) w->K[S][mu] = 0.0;
  for (int i = 0; i < n; i++)
    if (S & (1 << i))
      for (int mu = 0; mu < 4; mu++) w->K[S][mu] += q->k[i][mu];
  memset(w->J[S], 0, sizeof(w->J[S]));
  if (__builtin_popcount(S) == 1) {
    int i = __builtin_ctz(S);
    for (int mu = 0; mu < 4; mu++) w->J[S][col[i]][mu] = q->eps[i][mu];
    w->have[S] = 1;
    return;
  }
  const real g = q->g;
  cplx acc[8][4];
  memset(acc, 0, sizeof(acc));
  /* three-gluon vertex: unordered splits {S1, S2}; S1 holds the lowest member of S */
  const int low = S & (-S);
  for (int S1 = (S - 1) & S; S1 > 0; S1 = (S1 - 1) & S) {
    if (!(S1 & low)) continue;
    const int S2 = S ^ S1;
    dressed_current(q, col, S1, w);
    dressed_current(q, col, S2, w);
    for (int a = 0; a < 8; a++)
      for (int b = 0; b < 8; b++) {
        cplx t[4];
        vertex3(w->K[S1], w->J[S1][a], w->K[S2], w->J[S2][b], t);
        for (int c = 0; c < 8; c++) {
          const real f = FABC[a][b][c];
          if (f == 0.0) continue;
          /* (-i/P^2) * g f^{abc} V3 */
          for (int mu = 0; mu < 4; mu++) acc[c][mu] += -I * g * f * t[mu];
        }
      }
  }
  /* four-gluon vertex: unordered splits {S1, S2, S3}, legs (a,mu) (b,nu) (d,rho), out (c,sigma):
   *  -i g^2 [ f^{abe} f^{dce} (g^{mu rho} g^{nu sigma} - g^{mu sigma} g^{nu rho})
   *         + f^{ade} f^{bce} (g^{mu nu} g^{rho sigma} - g^{mu sigma} g^{nu rho})
   *         + f^{ace} f^{bde} (g^{mu nu} g^{rho sigma} - g^{mu rho} g^{nu sigma}) ] */
  for (int S1 = (S - 1) & S; S1 > 0; S1 = (S1 - 1) & S) {
    if (!(S1 & low)) continue;
    const int R = S ^ S1;
    const int low2 = R & (-R);
    for (int S2 = (R - 1) & R; S2 > 0; S2 = (S2 - 1) & R) {
      if (!(S2 & low2)) continue;
      const int S3 = R ^ S2;
      dressed_current(q, col, S1, w);
      dressed_current(q, col, S2, w);
      dressed_current(q, col, S3, w);
      for (int a = 0; a < 8; a++)
        for (int b = 0; b < 8; b++)
          for (int d = 0; d < 8; d++) {
            const cplx* j1 = w->J[S1][a];
            const cplx* j2 = w->J[S2][b];
            const cplx* j3 = w->J[S3][d];
            const cplx d12 = dot_cc(j1, j2), d13 = dot_cc(j1, j3), d23 = dot_cc(j2, j3);
            if (d12 == 0 && d13 == 0 && d23 == 0) continue;
            for (int c = 0; c < 8; c++) {
              real f1 = 0, f2 = 0, f3 = 0;
              for (int e = 0; e < 8; e++) {
                f1 += FABC[a][b][e] * FABC[d][c][e];
                f2 += FABC[a][d][e] * FABC[b][c][e];
                f3 += FABC[a][c][e] * FABC[b][d][e];
              }
              if (f1 == 0 && f2 == 0 && f3 == 0) continue;
              for (int mu = 0; mu < 4; mu++) {
                const cplx lor = f1 * (d13 * j2[mu] - d23 * j1[mu]) + f2 * (d12 * j3[mu] - d23 * j1[mu]) +
                                 f3 * (d12 * j3[mu] - d13 * j2[mu]);
                /* (-i/P^2) * (-i g^2) = -g^2 / P^2 */
                acc[c][mu] += -g * g * lor;
              }
            }
          }
    }
  }
  const real p2 = dot_rr(w->K[S], w->K[S]);
  for (int c = 0; c < 8; c++)
    for (int mu = 0; mu < 4; mu++) w->J[S][c][mu] = acc[c][mu] / p2;
  w->have[S] = 1;
}

/* sum over all external colours of |M|^2 for explicit external spin states */
int mgo_dressed_colour_sum(int n, const double* params, const double* kin, const double* eps, const double* pt,
                           const double* ubar, const double* ptb, const double* v, double* out) {
  qline q;
  int rc = fill_qline(&q, n, params, kin, eps, pt, ubar, ptb, v);
  if (rc) return rc;
  if (n > 4) return MGO_ERR_ARG;
  init_fabc();
  dressed_ws* w = (dressed_ws*)malloc(sizeof(dressed_ws));
  if (!w) return MGO_ERR_NOMEM;
  const int full = (1 << n) - 1;
  int col[MAXG];
  long total = 1;
  for (int i = 0; i < n; i++) total *= 8;
  real sum = 0.0;
  for (long code = 0; code < total; code++) {
    long c = code;
    for (int i = 0; i < n; i++) { col[i] = (int)(c % 8); c /= 8; }
    memset(w->have, 0, sizeof(w->have));
    /* quark row currents Psi[S][colour i_open][4] over gluon subsets S, built
     * from the top end: Psi[S] = sum_{B subset S} Psi[S\B] (i g Jslash^a(B) T^a) i(Qslash+m)/D */
    static __thread cplx Psi[1 << MAXG][3][3][4]; /* [S][i_top][open colour][spinor] */
    for (int it = 0; it < 3; it++)
      for (int jo = 0; jo < 3; jo++)
        for (int s4 = 0; s4 < 4; s4++) Psi[0][it][jo][s4] = (it == jo) ? q.ubar[s4] : 0.0;
    for (int S = 1; S < full; S++) {
      real Q[4];
      for (int mu = 0; mu < 4; mu++) Q[mu] = q.pt[mu];
      for (int i = 0; i < n; i++)
        if (S & (1 << i))
          for (int mu = 0; mu < 4; mu++) Q[mu] -= q.k[i][mu];
      const cplx den = dot_rr(Q, Q) - q.mt * q.mt + I * q.mt * q.wt;
      cplx P[4][4];
      slash_r(Q, P);
      for (int r = 0; r < 4; r++) P[r][r] += q.mt;
      cplx row[3][3][4];
      memset(row, 0, sizeof(row));
      for (int B = S; B > 0; B = (B - 1) & S) {
        const int A = S ^ B;
        dressed_current(&q, col, B, w);
        for (int a = 0; a < 8; a++) {
          cplx Sl[4][4];
          slash_c(w->J[B][a], Sl);
          for (int it = 0; it < 3; it++)
            for (int j = 0; j < 3; j++) {
              cplx t[4];
              rowmat(Psi[A][it][j], (const cplx(*)[4])Sl, t);
              for (int k = 0; k < 3; k++) {
                const cplx tc = TGEN[a][j][k];
                if (tc == 0) continue;
                for (int s4 = 0; s4 < 4; s4++) row[it][k][s4] += tc * t[s4];
              }
            }
        }
      }
      for (int it = 0; it < 3; it++)
        for (int k = 0; k < 3; k++) {
          cplx t[4];
          rowmat(row[it][k], (const cplx(*)[4])P, t);
          for (int s4 = 0; s4 < 4; s4++) Psi[S][it][k][s4] = (I * q.g) * (I / den) * t[s4];
        }
    }
    /* amplitude with open colours (i_top, j_antitop) */
    cplx M[3][3];
    memset(M, 0, sizeof(M));
    for (int B = full; B > 0; B = (B - 1) & full) {
      const int A = full ^ B;
      dressed_current(&q, col, B, w);
      for (int a = 0; a < 8; a++) {
        cplx Sl[4][4], t[4];
        slash_c(w->J[B][a], Sl);
        matcol((const cplx(*)[4])Sl, q.v, t);
        for (int it = 0; it < 3; it++)
          for (int j = 0; j < 3; j++) {
            const cplx r = rowcol(Psi[A][it][j], t);
            for (int k = 0; k < 3; k++) M[it][k] += (I * q.g) * TGEN[a][j][k] * r;
          }
      }
    }
    for (int it = 0; it < 3; it++)
      for (int k = 0; k < 3; k++) sum += creal(M[it][k] * conj(M[it][k]));
  }
  free(w);
  *out = sum;
  return MGO_OK;
}

/* ------------------------------------------------------------------ */
/* External-state test hooks                                           */
/* ------------------------------------------------------------------ */

static void to_double_c(const cplx* in, int n, double* out) {
  for (int i = 0; i < n; i++) {
    out[2 * i] = (double)creal(in[i]);
    out[2 * i + 1] = (double)cimag(in[i]);
  }
}

int mgo_spinor(int kind /*0 u, 1 v, 2 ubar, 3 vbar*/, const double* p, double m, int s, double* out) {
  cplx w[4], b[4];
  const real pr[4] = {p[0], p[1], p[2], p[3]};
  if (kind == 0 || kind == 2) spinor_u(pr, m, s, w);
  else spinor_v(pr, m, s, w);
  if (kind >= 2) {
    dirac_bar(w, b);
    to_double_c(b, 4, out);
  } else {
    to_double_c(w, 4, out);
  }
  return MGO_OK;
}

int mgo_polarisation(const double* k, int which, double* out) {
  const real kr[4] = {k[0], k[1], k[2], k[3]};
  real e[4];
  polarisation(kr, which, e);
  for (int i = 0; i < 4; i++) out[i] = (double)e[i];
  return MGO_OK;
}

int mgo_gamma(double* out /* complex [5][4][4]: gamma^0..3, gamma^5 */) {
  to_double_c(&GAM[0][0][0], 64, out);
  to_double_c(&GAM5[0][0], 16, out + 2 * 64);
  return MGO_OK;
}

/* ------------------------------------------------------------------ */
/* Full matrix elements                                                */
/* ------------------------------------------------------------------ */

/* e+(p1) e-(p2) -> mu+(p3) mu-(p4) through s-channel photon and Z */
static real me_eemumu(const oparams* o, const real* mom) {
  const real* p1 = mom;
  const real* p2 = mom + 4;
  const real* p3 = mom + 8;
  const real* p4 = mom + 12;
  const real alpha = 1.0 / o->alpha_em_inv;
  const real ee = sqrt(4.0 * PI_R * alpha);
  const real mz2 = o->mz * o->mz;
  const real mw2 = 0.5 * mz2 + sqrt(0.25 * mz2 * mz2 - PI_R * alpha * mz2 / (sqrt((real)2) * o->gf));
  const real sw2 = 1.0 - mw2 / mz2;
  const real cw2 = 1.0 - sw2;
  const real gl = -0.5 + sw2, gr = sw2;                /* T3 - Q sw^2 for Q = -1 */
  const real gz = ee / sqrt(sw2 * cw2);
  real ptot[4];
  for (int mu = 0; mu < 4; mu++) ptot[mu] = p1[mu] + p2[mu];
  const real s = dot_rr(ptot, ptot);
  const cplx prop_a = -I / s;
  const cplx prop_z = o->photon_only ? 0.0 : -I / (s - mz2 + I * o->mz * o->wz);
  /* Gamma_gamma^mu = -i e Q gamma^mu (Q = -1); Gamma_Z^mu = -i gz gamma^mu (gl PL + gr PR) */
  cplx PL[4][4], PR[4][4];
  for (int r = 0; r < 4; r++)
    for (int c = 0; c < 4; c++) {
      PL[r][c] = 0.5 * ((r == c ? 1.0 : 0.0) - GAM5[r][c]);
      PR[r][c] = 0.5 * ((r == c ? 1.0 : 0.0) + GAM5[r][c]);
    }
  cplx GA[4][4][4], GZ[4][4][4];
  for (int mu = 0; mu < 4; mu++) {
    cplx chir[4][4], tmp[4][4];
    for (int r = 0; r < 4; r++)
      for (int c = 0; c < 4; c++) chir[r][c] = gl * PL[r][c] + gr * PR[r][c];
    matmul4((const cplx(*)[4])GAM[mu], (const cplx(*)[4])chir, tmp);
    for (int r = 0; r < 4; r++)
      for (int c = 0; c < 4; c++) {
        GA[mu][r][c] = -I * ee * (-1.0) * GAM[mu][r][c];
        GZ[mu][r][c] = -I * gz * tmp[r][c];
      }
  }
  real sum = 0.0;
  for (int s1 = 0; s1 < 2; s1++)
    for (int s2 = 0; s2 < 2; s2++)
      for (int s3 = 0; s3 < 2; s3++)
        for (int s4 = 0; s4 < 2; s4++) {
          cplx v1[4], vb1[4], u2[4], v3[4], u4[4], ub4[4];
          spinor_v(p1, 0.0, s1, v1);
          dirac_bar(v1, vb1);
          spinor_u(p2, 0.0, s2, u2);
          spinor_v(p3, 0.0, s3, v3);
          spinor_u(p4, 0.0, s4, u4);
          dirac_bar(u4, ub4);
          cplx ja[4], jz[4], la[4], lz[4];
          for (int mu = 0; mu < 4; mu++) {
            cplx t[4];
            matcol((const cplx(*)[4])GA[mu], u2, t);
            ja[mu] = rowcol(vb1, t);
            matcol((const cplx(*)[4])GZ[mu], u2, t);
            jz[mu] = rowcol(vb1, t);
            matcol((const cplx(*)[4])GA[mu], v3, t);
            la[mu] = rowcol(ub4, t);
            matcol((const cplx(*)[4])GZ[mu], v3, t);
            lz[mu] = rowcol(ub4, t);
          }
          const cplx m = dot_cc(ja, la) * prop_a + dot_cc(jz, lz) * prop_z;
          sum += creal(m * conj(m));
        }
  return sum / 4.0;
}

/* u(p1) u~(p2) -> t(p3) t~(p4): the one s-channel gluon diagram,
 *   M = [vbar(p2) (i g gamma^mu T^a) u(p1)] (-i g_{mu nu} / s) [ubar(p3) (i g gamma^nu T^a) v(p4)],
 * with every colour index summed explicitly over the Gell-Mann generators
 * (colour factor sum_{ijkl} |sum_a T^a_{ji} T^a_{kl}|^2) and every spin state
 * summed with explicit Dirac-representation spinors.  IDEN = 4 spins x 9
 * colours. */
static real me_uutt(const oparams* o, const real* mom) {
  const real* p1 = mom;
  const real* p2 = mom + 4;
  const real* p3 = mom + 8;
  const real* p4 = mom + 12;
  const real g = sqrt(4.0 * PI_R * o->alpha_s);
  real ptot[4];
  for (int mu = 0; mu < 4; mu++) ptot[mu] = p1[mu] + p2[mu];
  const real s = dot_rr(ptot, ptot);
  real colour = 0.0;
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++)
      for (int k = 0; k < 3; k++)
        for (int l = 0; l < 3; l++) {
          cplx c = 0.0;
          for (int a = 0; a < 8; a++) c += TGEN[a][j][i] * TGEN[a][k][l];
          colour += creal(c * conj(c));
        }
  real sum = 0.0;
  for (int s1 = 0; s1 < 2; s1++)
    for (int s2 = 0; s2 < 2; s2++)
      for (int s3 = 0; s3 < 2; s3++)
        for (int s4 = 0; s4 < 2; s4++) {
          cplx u1[4], v2[4], vb2[4], u3[4], ub3[4], v4[4];
          spinor_u(p1, 0.0, s1, u1);
          spinor_v(p2, 0.0, s2, v2);
          dirac_bar(v2, vb2);
          spinor_u(p3, o->mt, s3, u3);
          dirac_bar(u3, ub3);
          spinor_v(p4, o->mt, s4, v4);
          cplx jl[4], jh[4];
          for (int mu = 0; mu < 4; mu++) {
            cplx t[4];
            matcol((const cplx(*)[4])GAM[mu], u1, t);
            jl[mu] = I * g * rowcol(vb2, t);
            matcol((const cplx(*)[4])GAM[mu], v4, t);
            jh[mu] = I * g * rowcol(ub3, t);
          }
          const cplx m = dot_cc(jl, jh) * (-I / s);
          sum += creal(m * conj(m));
        }
  return sum * colour / 36.0;
}

/* u(p1) u~(p2) -> t(p3) t~(p4) g(p5): the five diagrams written out with
 * explicit Dirac matrices (Feynman rules above; light quark massless):
 *   D1 gluon off the u line at the u end,  D2 at the u~ end,
 *   D3 off the top line at the t end,       D4 at the t~ end,
 *   D5 three-gluon vertex on the s-channel gluon.
 * Colour: each diagram's colour factor for every assignment (u i, u~ j, t k,
 * t~ l, gluon a) is an explicit sum over Gell-Mann generators and f^{abc}:
 *   D1 sum_b (T^b T^a)_{ji} T^b_{kl},  D2 sum_b (T^a T^b)_{ji} T^b_{kl},
 *   D3 sum_b T^b_{ji} (T^a T^b)_{kl},  D4 sum_b T^b_{ji} (T^b T^a)_{kl},
 *   D5 sum_{bc} f^{bca} T^b_{ji} T^c_{kl}.
 * IDEN = 4 spins x 9 colours. */
static cplx UUTTG_COL[5][3][3][3][3][8]; /* [diagram][i][j][k][l][a] */
static int uuttg_col_ready = 0;
static pthread_mutex_t uuttg_lock = PTHREAD_MUTEX_INITIALIZER;

static void init_uuttg_colour(void) {
  init_fabc();
  pthread_mutex_lock(&uuttg_lock);
  if (!uuttg_col_ready) {
    for (int i = 0; i < 3; i++)
      for (int j = 0; j < 3; j++)
        for (int k = 0; k < 3; k++)
          for (int l = 0; l < 3; l++)
            for (int a = 0; a < 8; a++) {
              cplx c[5] = {0, 0, 0, 0, 0};
              for (int b = 0; b < 8; b++) {
                cplx ba_ji = 0, ab_ji = 0, ab_kl = 0, ba_kl = 0;
                for (int m = 0; m < 3; m++) {
                  ba_ji += TGEN[b][j][m] * TGEN[a][m][i];
                  ab_ji += TGEN[a][j][m] * TGEN[b][m][i];
                  ab_kl += TGEN[a][k][m] * TGEN[b][m][l];
                  ba_kl += TGEN[b][k][m] * TGEN[a][m][l];
                }
                c[0] += ba_ji * TGEN[b][k][l];
                c[1] += ab_ji * TGEN[b][k][l];
                c[2] += TGEN[b][j][i] * ab_kl;
                c[3] += TGEN[b][j][i] * ba_kl;
                for (int cc = 0; cc < 8; cc++) c[4] += FABC[b][cc][a] * TGEN[b][j][i] * TGEN[cc][k][l];
              }
              for (int d = 0; d < 5; d++) UUTTG_COL[d][i][j][k][l][a] = c[d];
            }
    uuttg_col_ready = 1;
  }
  pthread_mutex_unlock(&uuttg_lock);
}

/* The five colour-stripped diagram values for fixed spins and a given
 * (complex) polarisation vector eps5 of the outgoing gluon (eps5 = k5 gives
 * the Ward identity). */
static void uuttg_diagrams(const oparams* o, const real* mom, int s1, int s2, int s3, int s4, const cplx eps5[4],
                           cplx A[5]) {
  const real* p1 = mom;
  const real* p2 = mom + 4;
  const real* p3 = mom + 8;
  const real* p4 = mom + 12;
  const real* p5 = mom + 16;
  const real g = sqrt(4.0 * PI_R * o->alpha_s);
  const real mt = o->mt;
  cplx u1[4], v2[4], vb2[4], u3[4], ub3[4], v4[4];
  spinor_u(p1, 0.0, s1, u1);
  spinor_v(p2, 0.0, s2, v2);
  dirac_bar(v2, vb2);
  spinor_u(p3, mt, s3, u3);
  dirac_bar(u3, ub3);
  spinor_v(p4, mt, s4, v4);
  cplx E[4][4];
  slash_c(eps5, E);
  real q34[4], s12[4], a[4], b[4], c[4], d[4];
  for (int mu = 0; mu < 4; mu++) {
    q34[mu] = p3[mu] + p4[mu];
    s12[mu] = p1[mu] + p2[mu];
    a[mu] = p1[mu] - p5[mu];   /* D1 light propagator */
    b[mu] = p5[mu] - p2[mu];   /* D2 light propagator (along the fermion flow) */
    c[mu] = p3[mu] + p5[mu];   /* D3 top propagator */
    d[mu] = -p4[mu] - p5[mu];  /* D4 top propagator (along the fermion flow) */
  }
  const real q2 = dot_rr(q34, q34), s = dot_rr(s12, s12);
  const cplx iw = I * mt * o->wt;
  /* propagator matrices: massless i qslash / q^2, top i (qslash + m) / (q^2 - m^2 + i m w) */
  cplx SA[4][4], SB[4][4], SC[4][4], SD[4][4];
  slash_r(a, SA);
  slash_r(b, SB);
  slash_r(c, SC);
  slash_r(d, SD);
  const cplx fa = I / dot_rr(a, a), fb = I / dot_rr(b, b);
  const cplx fc = I / (dot_rr(c, c) - mt * mt + iw), fd = I / (dot_rr(d, d) - mt * mt + iw);
  for (int r = 0; r < 4; r++)
    for (int cc = 0; cc < 4; cc++) {
      SA[r][cc] *= fa;
      SB[r][cc] *= fb;
      SC[r][cc] = (SC[r][cc] + (r == cc ? mt : 0.0)) * fc;
      SD[r][cc] = (SD[r][cc] + (r == cc ? mt : 0.0)) * fd;
    }
  const cplx ig = I * g;
  /* vertex-dressed spinors */
  cplx Eu1[4], SAEu1[4], vb2E[4], vb2ESB[4], ub3E[4], ub3ESC[4], Ev4[4], SDEv4[4];
  matcol((const cplx(*)[4])E, u1, Eu1);
  matcol((const cplx(*)[4])SA, Eu1, SAEu1);
  rowmat(vb2, (const cplx(*)[4])E, vb2E);
  rowmat(vb2E, (const cplx(*)[4])SB, vb2ESB);
  rowmat(ub3, (const cplx(*)[4])E, ub3E);
  rowmat(ub3E, (const cplx(*)[4])SC, ub3ESC);
  matcol((const cplx(*)[4])E, v4, Ev4);
  matcol((const cplx(*)[4])SD, Ev4, SDEv4);
  cplx L[4], H[4], L1[4], L2[4], H3[4], H4[4];
  for (int mu = 0; mu < 4; mu++) {
    cplx t[4];
    matcol((const cplx(*)[4])GAM[mu], u1, t);
    L[mu] = ig * rowcol(vb2, t);                  /* vbar2 (i g gamma^mu) u1 */
    L2[mu] = ig * ig * rowcol(vb2ESB, t);         /* vbar2 (ig eps) S_B (ig gamma^mu) u1 */
    matcol((const cplx(*)[4])GAM[mu], SAEu1, t);
    L1[mu] = ig * ig * rowcol(vb2, t);            /* vbar2 (ig gamma^mu) S_A (ig eps) u1 */
    matcol((const cplx(*)[4])GAM[mu], v4, t);
    H[mu] = ig * rowcol(ub3, t);                  /* ubar3 (i g gamma^mu) v4 */
    H3[mu] = ig * ig * rowcol(ub3ESC, t);         /* ubar3 (ig eps) S_C (ig gamma^mu) v4 */
    matcol((const cplx(*)[4])GAM[mu], SDEv4, t);
    H4[mu] = ig * ig * rowcol(ub3, t);            /* ubar3 (ig gamma^mu) S_D (ig eps) v4 */
  }
  /* gluon propagators -i g_{mu nu} / k^2 */
  A[0] = dot_cc(L1, H) * (-I / q2);
  A[1] = dot_cc(L2, H) * (-I / q2);
  A[2] = dot_cc(L, H3) * (-I / s);
  A[3] = dot_cc(L, H4) * (-I / s);
  /* three-gluon vertex with incoming (b, mu, P = p1 + p2), (c, nu, -q34),
   * (a, rho, -p5): g [g^{mu nu}(P + q34)^rho + g^{nu rho}(p5 - q34)^mu
   * + g^{rho mu}(-p5 - P)^nu], times f^{bca} (in the colour factor) */
  const cplx GL[4] = {L[0] * (-I / s), L[1] * (-I / s), L[2] * (-I / s), L[3] * (-I / s)};
  const cplx GH[4] = {H[0] * (-I / q2), H[1] * (-I / q2), H[2] * (-I / q2), H[3] * (-I / q2)};
  real x[4], y[4], z[4];
  for (int mu = 0; mu < 4; mu++) {
    x[mu] = s12[mu] + q34[mu];
    y[mu] = p5[mu] - q34[mu];
    z[mu] = -p5[mu] - s12[mu];
  }
  A[4] = g * (dot_cc(GL, GH) * dot_rc(x, eps5) + dot_cc(GH, eps5) * dot_rc(y, GL) + dot_cc(eps5, GL) * dot_rc(z, GH));
}

static real me_uuttg(const oparams* o, const real* mom) {
  init_uuttg_colour();
  real sum = 0.0;
  for (int s1 = 0; s1 < 2; s1++)
    for (int s2 = 0; s2 < 2; s2++)
      for (int s3 = 0; s3 < 2; s3++)
        for (int s4 = 0; s4 < 2; s4++)
          for (int pol = 0; pol < 2; pol++) {
            real e[4];
            polarisation(mom + 16, pol, e);
            const cplx eps[4] = {e[0], e[1], e[2], e[3]};
            cplx A[5];
            uuttg_diagrams(o, mom, s1, s2, s3, s4, eps, A);
            for (int i = 0; i < 3; i++)
              for (int j = 0; j < 3; j++)
                for (int k = 0; k < 3; k++)
                  for (int l = 0; l < 3; l++)
                    for (int a = 0; a < 8; a++) {
                      cplx m = 0;
                      for (int dg = 0; dg < 5; dg++) m += UUTTG_COL[dg][i][j][k][l][a] * A[dg];
                      sum += creal(m * conj(m));
                    }
          }
  return sum / 36.0;
}

/* Colour-dressed amplitudes of u u~ -> t t~ g for given spins and a complex
 * gluon polarisation vector: out[(((i*3+j)*3+k)*3+l)*8+a] (complex
 * interleaved, 648 entries).  Test hook (Ward identity: eps5 = k5). */
int mgo_uuttg_amps(const double* params, const double* mom, int s1, int s2, int s3, int s4,
                   const double* eps5 /* complex [4] */, double* out) {
  oparams o;
  unpack_params(params, &o);
  init_uuttg_colour();
  real p[20];
  for (int i = 0; i < 20; i++) p[i] = mom[i];
  cplx e[4];
  for (int mu = 0; mu < 4; mu++) e[mu] = eps5[2 * mu] + I * eps5[2 * mu + 1];
  cplx A[5];
  uuttg_diagrams(&o, p, s1, s2, s3, s4, e, A);
  int n = 0;
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++)
      for (int k = 0; k < 3; k++)
        for (int l = 0; l < 3; l++)
          for (int a = 0; a < 8; a++) {
            cplx m = 0;
            for (int dg = 0; dg < 5; dg++) m += UUTTG_COL[dg][i][j][k][l][a] * A[dg];
            out[2 * n] = (double)creal(m);
            out[2 * n + 1] = (double)cimag(m);
            n++;
          }
  return MGO_OK;
}

/* ------------------------------------------------------------------ */
/* u u~ -> t t~ + n gluons (n <= 2): colour-dressed Berends-Giele       */
/* recursion over both quark lines                                    */
/* ------------------------------------------------------------------ */

/* Legs: 0 u (incoming, the root of the recursion), 1 u~ (incoming), 2 t, 3 t~,
 * 4.. gluons (outgoing).  Off-shell currents are built over subsets S of the
 * legs 1.. (bit leg-1), with the Feynman rules of the header:
 *   gluon current  J^c(S)    no u~, both or neither of t, t~: the three- and
 *                            four-gluon vertices, and the top line closed by
 *                            i g gamma^mu T^c;  times -i/P^2
 *   light row      Ubar_m(S) holds u~ (and possibly the closed top line)
 *   top row        Tbar_m(S) holds t,  top column T_m(S) holds t~
 *   quark propagator i (Qslash + m) / (Q^2 - m^2 + i m Gamma) (top), i Qslash/Q^2 (u)
 * Each current carries its off-shell colour (c < 8 or m < 3) and, as a plain
 * array index x = 9 j + 3 k + l, the colours j, k, l of the external u~, t,
 * t~; a current that does not hold one of those legs is the same for every
 * value of its index, so products of two currents are taken entrywise in x.
 * The amplitude M[i][x] for the u colour i closes at the root:
 *   M = sum_{A u B} Ubar_m(A) (i g Jslash^c(B) T^c_{m i}) u(p1).
 * The gluon colours are fixed per evaluation and summed outside. */
#define QQ_LEGS 6
#define QQ_X 27
typedef struct {
  cplx v[8][QQ_X][4];
  int have, nz; /* computed; some entry non-zero */
} qq_cur;

typedef struct {
  int nleg;                 /* legs 1 .. nleg-1 below the root            */
  real g, mt, wt;
  real kin[QQ_LEGS][4];     /* incoming momentum of each leg              */
  cplx eps[QQ_LEGS][4];     /* gluon polarisations (legs >= 4)            */
  int col[QQ_LEGS];         /* gluon colours (legs >= 4)                  */
  cplx u1[4], vb2[4], ub3[4], v4[4];
  qq_cur c[1 << (QQ_LEGS - 1)];
} qq_ws;

static int qq_kind(int S) {
  /* 1 gluon, 2 light row, 3 top row, 4 top column, 0 none */
  const int has1 = S & 1, has2 = (S >> 1) & 1, has3 = (S >> 2) & 1;
  if (!has1 && has2 == has3) return 1;
  if (has1 && has2 == has3) return 2;
  if (!has1 && has2 && !has3) return 3;
  if (!has1 && !has2 && has3) return 4;
  return 0;
}

static void qq_momentum(const qq_ws* w, int S, real K[4]) {
  for (int mu = 0; mu < 4; mu++) K[mu] = 0.0;
  for (int b = 0; b < w->nleg - 1; b++)
    if (S & (1 << b))
      for (int mu = 0; mu < 4; mu++) K[mu] += w->kin[b + 1][mu];
}

static void qq_current(qq_ws* w, int S);

/* row (off-shell colour m) times i g Jslash^c T^c_{m n}, summed over c, m, into acc[n][x] */
static void qq_row_times_gluon(const qq_cur* R, const qq_cur* G, const real g, cplx acc[3][QQ_X][4]) {
  for (int c = 0; c < 8; c++)
    for (int x = 0; x < QQ_X; x++) {
      const cplx* j = G->v[c][x];
      if (j[0] == 0 && j[1] == 0 && j[2] == 0 && j[3] == 0) continue;
      cplx Sl[4][4];
      slash_c(j, Sl);
      for (int m = 0; m < 3; m++) {
        const cplx* r = R->v[m][x];
        if (r[0] == 0 && r[1] == 0 && r[2] == 0 && r[3] == 0) continue;
        cplx t[4];
        rowmat(r, (const cplx(*)[4])Sl, t);
        for (int n = 0; n < 3; n++) {
          const cplx tc = TGEN[c][m][n];
          if (tc == 0) continue;
          for (int s = 0; s < 4; s++) acc[n][x][s] += I * g * tc * t[s];
        }
      }
    }
}

static void qq_current(qq_ws* w, int S) {
  qq_cur* cur = &w->c[S];
  if (cur->have) return;
  cur->have = 1;
  const int kind = qq_kind(S);
  memset(cur->v, 0, (kind == 1 ? 8 : 3) * sizeof(cur->v[0]));
  const int low = S & (-S);
  const real g = w->g;
  if (__builtin_popcount(S) == 1) {
    const int leg = __builtin_ctz(S) + 1;
    for (int x = 0; x < QQ_X; x++) {
      const int j = x / 9, k = (x / 3) % 3, l = x % 3;
      for (int s = 0; s < 4; s++) {
        if (leg == 1) cur->v[j][x][s] = w->vb2[s];
        else if (leg == 2) cur->v[k][x][s] = w->ub3[s];
        else if (leg == 3) cur->v[l][x][s] = w->v4[s];
        else cur->v[w->col[leg]][x][s] = w->eps[leg][s];
      }
    }
    cur->nz = 1;
    return;
  }
  real K[4];
  qq_momentum(w, S, K);
  if (kind == 1) {
    cplx acc[8][QQ_X][4]; /* per recursion level: sub-currents are built inside the loops */
    memset(acc, 0, sizeof(acc));
    /* three-gluon vertex, unordered pairs of gluon currents */
    for (int A = (S - 1) & S; A > 0; A = (A - 1) & S) {
      if (!(A & low)) continue;
      const int B = S ^ A;
      if (qq_kind(A) != 1 || qq_kind(B) != 1) continue;
      qq_current(w, A);
      qq_current(w, B);
      if (!w->c[A].nz || !w->c[B].nz) continue;
      real KA[4], KB[4];
      qq_momentum(w, A, KA);
      qq_momentum(w, B, KB);
      for (int a = 0; a < 8; a++)
        for (int b = 0; b < 8; b++) {
          int any = 0;
          for (int c = 0; c < 8; c++) any |= FABC[a][b][c] != 0.0;
          if (!any) continue;
          for (int x = 0; x < QQ_X; x++) {
            const cplx* ja = w->c[A].v[a][x];
            const cplx* jb = w->c[B].v[b][x];
            if ((ja[0] == 0 && ja[1] == 0 && ja[2] == 0 && ja[3] == 0) ||
                (jb[0] == 0 && jb[1] == 0 && jb[2] == 0 && jb[3] == 0))
              continue;
            cplx t[4];
            vertex3(KA, ja, KB, jb, t);
            for (int c = 0; c < 8; c++) {
              const real f = FABC[a][b][c];
              if (f == 0.0) continue;
              for (int mu = 0; mu < 4; mu++) acc[c][x][mu] += -I * g * f * t[mu]; /* (-i/P^2) g f V3 */
            }
          }
        }
    }
    /* four-gluon vertex, unordered triples of gluon currents (as in the
     * one-line colour-dressed recursion above) */
    for (int A = (S - 1) & S; A > 0; A = (A - 1) & S) {
      if (!(A & low)) continue;
      const int R = S ^ A;
      const int low2 = R & (-R);
      for (int B = (R - 1) & R; B > 0; B = (B - 1) & R) {
        if (!(B & low2)) continue;
        const int C = R ^ B;
        if (qq_kind(A) != 1 || qq_kind(B) != 1 || qq_kind(C) != 1) continue;
        qq_current(w, A);
        qq_current(w, B);
        qq_current(w, C);
        for (int a = 0; a < 8; a++)
          for (int b = 0; b < 8; b++)
            for (int d = 0; d < 8; d++)
              for (int x = 0; x < QQ_X; x++) {
                const cplx* j1 = w->c[A].v[a][x];
                const cplx* j2 = w->c[B].v[b][x];
                const cplx* j3 = w->c[C].v[d][x];
                const cplx d12 = dot_cc(j1, j2), d13 = dot_cc(j1, j3), d23 = dot_cc(j2, j3);
                if (d12 == 0 && d13 == 0 && d23 == 0) continue;
                for (int c = 0; c < 8; c++) {
                  real f1 = 0, f2 = 0, f3 = 0;
                  for (int e = 0; e < 8; e++) {
                    f1 += FABC[a][b][e] * FABC[d][c][e];
                    f2 += FABC[a][d][e] * FABC[b][c][e];
                    f3 += FABC[a][c][e] * FABC[b][d][e];
                  }
                  if (f1 == 0 && f2 == 0 && f3 == 0) continue;
                  for (int mu = 0; mu < 4; mu++) {
                    const cplx lor = f1 * (d13 * j2[mu] - d23 * j1[mu]) + f2 * (d12 * j3[mu] - d23 * j1[mu]) +
                                     f3 * (d12 * j3[mu] - d13 * j2[mu]);
                    acc[c][x][mu] += -g * g * lor; /* (-i/P^2) (-i g^2) */
                  }
                }
              }
      }
    }
    /* the top line closed into the gluon: Tbar_m(A) (i g gamma^mu T^c_{mn}) T_n(B) */
    if (S & 2) {
      for (int A = (S - 1) & S; A > 0; A = (A - 1) & S) {
        const int B = S ^ A;
        if (qq_kind(A) != 3 || qq_kind(B) != 4) continue;
        qq_current(w, A);
        qq_current(w, B);
        for (int x = 0; x < QQ_X; x++)
          for (int m = 0; m < 3; m++)
            for (int n = 0; n < 3; n++) {
              const cplx* r = w->c[A].v[m][x];
              const cplx* cc = w->c[B].v[n][x];
              for (int mu = 0; mu < 4; mu++) {
                cplx t[4];
                matcol((const cplx(*)[4])GAM[mu], cc, t);
                const cplx rv = rowcol(r, t);
                if (rv == 0) continue;
                for (int c = 0; c < 8; c++) {
                  const cplx tc = TGEN[c][m][n];
                  if (tc != 0) acc[c][x][mu] += g * tc * rv; /* (-i/P^2) (i g) */
                }
              }
            }
      }
    }
    const real p2 = dot_rr(K, K);
    int nz = 0;
    for (int c = 0; c < 8; c++)
      for (int x = 0; x < QQ_X; x++)
        for (int mu = 0; mu < 4; mu++) {
          cur->v[c][x][mu] = acc[c][x][mu] / p2;
          nz |= acc[c][x][mu] != 0;
        }
    cur->nz = nz;
    return;
  }
  /* quark lines: the leg at the line's end plus gluon currents attached */
  cplx acc3[3][QQ_X][4];
  memset(acc3, 0, sizeof(acc3));
  const int end = (kind == 2) ? 1 : (kind == 3) ? 2 : 4; /* bit of the line's external leg */
  real Q[4];
  for (int A = (S - 1) & S; A > 0; A = (A - 1) & S) {
    if (!(A & end)) continue;
    const int B = S ^ A;
    if (qq_kind(A) != kind || qq_kind(B) != 1) continue;
    qq_current(w, A);
    qq_current(w, B);
    if (!w->c[A].nz || !w->c[B].nz) continue;
    if (kind != 4) {
      qq_row_times_gluon(&w->c[A], &w->c[B], g, acc3);
    } else {
      /* column: T^c_{m n} (i g Jslash^c) T_n(A) */
      for (int c = 0; c < 8; c++)
        for (int x = 0; x < QQ_X; x++) {
          const cplx* j = w->c[B].v[c][x];
          if (j[0] == 0 && j[1] == 0 && j[2] == 0 && j[3] == 0) continue;
          cplx Sl[4][4];
          slash_c(j, Sl);
          for (int n = 0; n < 3; n++) {
            cplx t[4];
            matcol((const cplx(*)[4])Sl, w->c[A].v[n][x], t);
            for (int m = 0; m < 3; m++) {
              const cplx tc = TGEN[c][m][n];
              if (tc == 0) continue;
              for (int s = 0; s < 4; s++) acc3[m][x][s] += I * g * tc * t[s];
            }
          }
        }
    }
  }
  /* propagator momentum along the fermion flow: rows end at t (p3) or at the
   * incoming u~ (-p2), columns start at the outgoing t~ (-p4); every attached
   * current adds its incoming momentum with the sign of the flow */
  const real* kend = w->kin[__builtin_ctz(end) + 1];
  for (int mu = 0; mu < 4; mu++) {
    const real attached = K[mu] - kend[mu];
    Q[mu] = (kind == 4) ? (kend[mu] + attached) : (-kend[mu] - attached);
  }
  const real m = (kind == 2) ? 0.0 : w->mt;
  const cplx den = dot_rr(Q, Q) - m * m + ((kind == 2) ? 0.0 : I * m * w->wt);
  cplx P[4][4];
  slash_r(Q, P);
  for (int r = 0; r < 4; r++) P[r][r] += m;
  int nz = 0;
  for (int c = 0; c < 3; c++)
    for (int x = 0; x < QQ_X; x++) {
      cplx t[4];
      if (kind == 4) matcol((const cplx(*)[4])P, acc3[c][x], t);
      else rowmat(acc3[c][x], (const cplx(*)[4])P, t);
      for (int s = 0; s < 4; s++) {
        cur->v[c][x][s] = (I / den) * t[s];
        nz |= t[s] != 0;
      }
    }
  cur->nz = nz;
}

/* sum over all external colours of |M|^2 for the spin states and gluon
 * polarisations set in w (the gluon colours are summed here) */
static real qq_colour_sum(qq_ws* w) {
  const int ng = w->nleg - 4;
  const int full = (1 << (w->nleg - 1)) - 1;
  int ncol = 1;
  for (int i = 0; i < ng; i++) ncol *= 8;
  real sum = 0.0;
  for (int code = 0; code < ncol; code++) {
    int cc = code;
    for (int i = 0; i < ng; i++) {
      w->col[4 + i] = cc % 8;
      cc /= 8;
    }
    for (int S = 0; S <= full; S++) w->c[S].have = 0;
    cplx M[3][QQ_X];
    memset(M, 0, sizeof(M));
    for (int A = full; A > 0; A = (A - 1) & full) {
      if (!(A & 1)) continue;
      const int B = full ^ A;
      if (B == 0 || qq_kind(A) != 2 || qq_kind(B) != 1) continue;
      qq_current(w, A);
      qq_current(w, B);
      cplx acc[3][QQ_X][4];
      memset(acc, 0, sizeof(acc));
      qq_row_times_gluon(&w->c[A], &w->c[B], w->g, acc);
      for (int i = 0; i < 3; i++)
        for (int x = 0; x < QQ_X; x++) M[i][x] += rowcol(acc[i][x], w->u1);
    }
    for (int i = 0; i < 3; i++)
      for (int x = 0; x < QQ_X; x++) sum += creal(M[i][x] * conj(M[i][x]));
  }
  return sum;
}

/* u(p1) u~(p2) -> t(p3) t~(p4) + ng gluons (p5, p6): every spin state of the
 * quarks (Dirac-representation spin-z spinors) and every linear polarisation
 * of the gluons, every colour; IDEN = 4 spins x 9 colours x ng!.  If eps_in
 * is not NULL it replaces the gluon polarisations (complex [ng][4], one spin
 * state of the gluons) and the result is the sum over quark spins only. */
static real me_uutt_ng(const oparams* o, int ng, const real* mom, const cplx* eps_in) {
  if (ng < 0 || ng > 2) return NAN;
  init_fabc();
  qq_ws* w = (qq_ws*)malloc(sizeof(qq_ws));
  if (!w) return NAN;
  w->nleg = 4 + ng;
  w->g = sqrt(4.0 * PI_R * o->alpha_s);
  w->mt = o->mt;
  w->wt = o->wt;
  for (int mu = 0; mu < 4; mu++) {
    w->kin[0][mu] = mom[mu];
    w->kin[1][mu] = mom[4 + mu];
    w->kin[2][mu] = -mom[8 + mu];
    w->kin[3][mu] = -mom[12 + mu];
    for (int i = 0; i < ng; i++) w->kin[4 + i][mu] = -mom[16 + 4 * i + mu];
  }
  real pol[2][2][4];
  for (int i = 0; i < ng; i++) {
    polarisation(mom + 16 + 4 * i, 0, pol[i][0]);
    polarisation(mom + 16 + 4 * i, 1, pol[i][1]);
  }
  real sum = 0.0;
  const int npol = eps_in ? 1 : (1 << ng);
  for (int s = 0; s < 16; s++) {
    cplx v2[4], u3[4];
    spinor_u(mom, 0.0, s & 1, w->u1);
    spinor_v(mom + 4, 0.0, (s >> 1) & 1, v2);
    dirac_bar(v2, w->vb2);
    spinor_u(mom + 8, o->mt, (s >> 2) & 1, u3);
    dirac_bar(u3, w->ub3);
    spinor_v(mom + 12, o->mt, (s >> 3) & 1, w->v4);
    for (int h = 0; h < npol; h++) {
      for (int i = 0; i < ng; i++)
        for (int mu = 0; mu < 4; mu++)
          w->eps[4 + i][mu] = eps_in ? eps_in[4 * i + mu] : (cplx)pol[i][(h >> i) & 1][mu];
      sum += qq_colour_sum(w);
    }
  }
  free(w);
  if (eps_in) return sum;
  real iden = 36.0;
  for (int i = 2; i <= ng; i++) iden *= i;
  return sum / iden;
}

/* Test hook: |M|^2 summed over quark spins and all colours for given complex
 * gluon polarisations eps[ng][4] (interleaved re, im); eps = k gives the Ward
 * identity. */
int mgo_uutt_ng_fixed_pol(int ng, const double* params, const double* mom, const double* eps, double* out) {
  if (ng < 1 || ng > 2) return MGO_ERR_ARG;
  oparams o;
  unpack_params(params, &o);
  real p[4 * QQ_LEGS];
  for (int i = 0; i < 4 * (4 + ng); i++) p[i] = mom[i];
  cplx e[2 * 4];
  for (int i = 0; i < 4 * ng; i++) e[i] = eps[2 * i] + I * eps[2 * i + 1];
  *out = (double)me_uutt_ng(&o, ng, p, e);
  return MGO_OK;
}

/* Test hook: the two-line recursion for 0, 1 or 2 gluons (the 0- and 1-gluon
 * cases are evaluated independently by me_uutt and me_uuttg). */
int mgo_uutt_ng(int ng, const double* params, const double* mom, int64_t nevt, double* me) {
  if (ng < 0 || ng > 2 || nevt < 0) return MGO_ERR_ARG;
  oparams o;
  unpack_params(params, &o);
  const int npar = 4 + ng;
  for (int64_t e = 0; e < nevt; e++) {
    real p[4 * QQ_LEGS];
    for (int i = 0; i < 4 * npar; i++) p[i] = mom[(size_t)e * npar * 4 + i];
    me[e] = (double)me_uutt_ng(&o, ng, p, NULL);
  }
  return MGO_OK;
}

/* g(p1) g(p2) -> t(p3) t~(p4) g(p5) ... : n gluons in total.
 * flow_w (may be NULL): sum over spin states of |A(sigma)|^2 per ordering. */
static real me_ggtt_ng_w(const oparams* o, int n, const real* mom, real* flow_w);
static real me_ggtt_ng(const oparams* o, int n, const real* mom) { return me_ggtt_ng_w(o, n, mom, NULL); }
static real me_ggtt_ng_w(const oparams* o, int n, const real* mom, real* flow_w) {
  const cplx* C = colour_matrix(n);
  if (!C) return NAN;
  const int np = factorial(n);
  /* gluon index -> particle slot; initial gluons 0,1 then final gluons 4.. */
  int slot[MAXG];
  slot[0] = 0;
  slot[1] = 1;
  for (int i = 2; i < n; i++) slot[i] = i + 2;
  qline q;
  q.n = n;
  q.g = sqrt(4.0 * PI_R * o->alpha_s);
  q.mt = o->mt;
  q.wt = o->wt;
  for (int mu = 0; mu < 4; mu++) {
    q.pt[mu] = mom[8 + mu];
    q.ptb[mu] = mom[12 + mu];
  }
  real pol[MAXG][2][4];
  for (int i = 0; i < n; i++) {
    const real* p = mom + 4 * slot[i];
    const real sign = (slot[i] < 2) ? 1.0 : -1.0; /* incoming momentum */
    for (int mu = 0; mu < 4; mu++) q.k[i][mu] = sign * p[mu];
    polarisation(p, 0, pol[i][0]);
    polarisation(p, 1, pol[i][1]);
  }
  cplx ubar_s[2][4], v_s[2][4];
  for (int s = 0; s < 2; s++) {
    cplx u[4];
    spinor_u(q.pt, o->mt, s, u);
    dirac_bar(u, ubar_s[s]);
    spinor_v(q.ptb, o->mt, s, v_s[s]);
  }
  real sum = 0.0;
  cplx A[MAXPERM];
  const int nhel = 1 << (n + 2);
  if (flow_w)
    for (int i = 0; i < np; i++) flow_w[i] = 0;
  for (int h = 0; h < nhel; h++) {
    for (int i = 0; i < n; i++)
      for (int mu = 0; mu < 4; mu++) q.eps[i][mu] = pol[i][(h >> i) & 1][mu]; /* real: eps* = eps */
    const int st = (h >> n) & 1, stb = (h >> (n + 1)) & 1;
    for (int c = 0; c < 4; c++) {
      q.ubar[c] = ubar_s[st][c];
      q.v[c] = v_s[stb][c];
    }
    all_ordered_amplitudes(&q, A);
    cplx s = 0;
    for (int i = 0; i < np; i++)
      for (int j = 0; j < np; j++) s += conj(A[i]) * C[i * np + j] * A[j];
    sum += creal(s);
    if (flow_w)
      for (int i = 0; i < np; i++) flow_w[i] += creal(A[i] * conj(A[i]));
  }
  real iden = 4.0 * 64.0;
  for (int i = 2; i <= n - 2; i++) iden *= i; /* identical final-state gluons */
  return sum / iden;
}

static int proc_gluons(int proc) {
  switch (proc) {
    case MGO_GGTT: return 2;
    case MGO_GGTTG: return 3;
    case MGO_GGTTGG: return 4;
    case MGO_GGTTGGG: return 5;
    default: return 0;
  }
}

int mgo_npar(int proc) {
  if (proc == MGO_EEMUMU || proc == MGO_UUTT) return 4;
  if (proc == MGO_UUTTG) return 5;
  if (proc == MGO_UUTTGG) return 6;
  const int n = proc_gluons(proc);
  return n ? n + 2 : MGO_ERR_ARG;
}

/* Colour-flow weights w[i][sigma] = sum over spin states of |A(sigma)|^2
 * (orderings lexicographic) for g g -> t t~ + gluons; the event-by-event
 * choice of a leading colour flow draws sigma with probability w / sum w. */
int mgo_flow_weights(int proc, const double* params, const double* mom, int64_t nevt, double* w) {
  oparams o;
  unpack_params(params, &o);
  const int n = proc_gluons(proc);
  if (!n || nevt < 0) return MGO_ERR_ARG;
  if (!colour_matrix(n)) return MGO_ERR_NOMEM;
  const int npar = n + 2, np = factorial(n);
  for (int64_t e = 0; e < nevt; e++) {
    real p[4 * (MAXG + 2)], fw[MAXPERM];
    for (int i = 0; i < npar * 4; i++) p[i] = mom[(size_t)e * npar * 4 + i];
    me_ggtt_ng_w(&o, n, p, fw);
    for (int i = 0; i < np; i++) w[(size_t)e * np + i] = (double)fw[i];
  }
  return MGO_OK;
}

/* me[i] for events i in [0, nevt): mom = [nevt][npar][4] */
int mgo_me(int proc, const double* params, const double* mom, int64_t nevt, double* me) {
  oparams o;
  unpack_params(params, &o);
  const int npar = mgo_npar(proc);
  if (npar < 0 || nevt < 0) return MGO_ERR_ARG;
  if (proc_gluons(proc) && !colour_matrix(proc_gluons(proc))) return MGO_ERR_NOMEM;
  for (int64_t e = 0; e < nevt; e++) {
    real p[4 * (MAXG + 2)];
    for (int i = 0; i < npar * 4; i++) p[i] = mom[(size_t)e * npar * 4 + i];
    me[e] = (double)((proc == MGO_EEMUMU) ? me_eemumu(&o, p)
                     : (proc == MGO_UUTT) ? me_uutt(&o, p)
                     : (proc == MGO_UUTTG) ? me_uuttg(&o, p)
                     : (proc == MGO_UUTTGG) ? me_uutt_ng(&o, 2, p, NULL)
                                           : me_ggtt_ng(&o, proc_gluons(proc), p));
  }
  return MGO_OK;
}
