/*
 * oracle.c -- plain, slow FP64 reference of the multideterminant evaluation.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library. The product path never calls it.
 * It shares no code, header or table with the CUDA library.
 *
 * What it computes is the definition, not the fast method:
 *   Psi(R) = sum_k c_k Det S^up_k(R_up) Det S^dn_k(R_dn)        (Eq. 1)
 * where [S^s_k]_{i a} = phi_{o_a}(r_i) with the occupied orbitals o_a of the
 * spin-determinant taken in ascending order (Sec. 2.1 bit-string encoding).
 * Every distinct spin determinant gets its full Slater matrix, an LU
 * factorisation with partial pivoting (the dgetrf route of Sec. 2.2), and its
 * derivatives by cofactors: since row i of S depends only on r_i,
 *   d_{i,mu} Det S = sum_a d_mu phi_{o_a}(r_i) cof_{i a}(S),
 *   cof_{i a}(S) = Det S * (S^-1)_{a i},
 * for mu = x, y, z and the Laplacian (Sec. 2.3, Eqs. 5-8; Eq. 8 read with the
 * inverse indexed (a, i)). The gradient and Laplacian of Psi are then summed
 * over the product list (Eqs. 5-7; the Eq. 6 cross terms are zero because no
 * electron belongs to both spin blocks). Orbitals are contracted Cartesian
 * Gaussians x^a y^b z^c sum_p d_p exp(-alpha_p r^2) combined by the AO->MO
 * matrix (Sec. 2, first paragraph). Sums use Neumaier compensated summation.
 * Local energy: E_L = -1/2 sum_i Lap_i Psi / Psi + V (Sec. 4, one MC step
 * computes Psi, the drift and E_L).
 *
 * Compile: gcc -O2 -ffp-contract=off -fPIC -shared oracle.c -lm -lpthread
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXL 3

/* ------------------------------------------------------------------------ */
/* Neumaier compensated summation                                            */
typedef struct { double s, c; } nsum;
static inline void nadd(nsum* a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x; else a->c += (x - t) + a->s;
  a->s = t;
}
static inline double nval(const nsum* a) { return a->s + a->c; }

static double ipow(double x, int n) { double r = 1.0; for (int i = 0; i < n; i++) r *= x; return r; }

/* Number of Cartesian components of a shell of angular momentum l. */
static int ncart(int l) { return (l + 1) * (l + 2) / 2; }

/* Component c of a shell of angular momentum l: exponents (a, b, c) in the
 * order xx, xy, xz, yy, yz, zz (a descending, then b descending). */
static void cart_exponents(int l, int idx, int* ea, int* eb, int* ec) {
  int n = 0;
  for (int a = l; a >= 0; a--)
    for (int b = l - a; b >= 0; b--) {
      if (n == idx) { *ea = a; *eb = b; *ec = l - a - b; return; }
      n++;
    }
}

int oracle_n_ao(int n_shell, const int* shell_l) {
  int n = 0;
  for (int s = 0; s < n_shell; s++) n += ncart(shell_l[s]);
  return n;
}

/* One Cartesian factor t^e and its first and second derivatives. */
static void pow_d(double t, int e, double* f, double* d1, double* d2) {
  *f = ipow(t, e);
  *d1 = e >= 1 ? e * ipow(t, e - 1) : 0.0;
  *d2 = e >= 2 ? e * (e - 1) * ipow(t, e - 2) : 0.0;
}

/*
 * AO values and derivatives at n_pts points.
 * out[p][0..4][mu] = chi_mu, d/dx, d/dy, d/dz, Laplacian.
 * Each primitive g = x^a y^b z^c exp(-alpha r^2) factorises into three 1-D
 * factors X(x) Y(y) Z(z) with X = x^a exp(-alpha x^2), so
 *   dg/dx = X' Y Z,   Lap g = X'' Y Z + X Y'' Z + X Y Z''
 *   X'  = (a x^(a-1) - 2 alpha x^(a+1)) e,  X'' = (a(a-1) x^(a-2) - 2 alpha (2a+1) x^a + 4 alpha^2 x^(a+2)) e.
 */
int oracle_ao_eval(int n_shell, const int* shell_l, const int* shell_center,
                   const int* shell_nprim, const double* alpha, const double* coef,
                   const double* nuc_xyz, int n_pts, const double* pts, double* out) {
  int n_ao = oracle_n_ao(n_shell, shell_l);
  for (int p = 0; p < n_pts; p++) {
    double* o = out + (size_t)p * 5 * n_ao;
    int mu = 0, prim = 0;
    for (int s = 0; s < n_shell; s++) {
      int l = shell_l[s];
      if (l < 0 || l > ORC_MAXL) return -1;
      const double* C = nuc_xyz + 3 * shell_center[s];
      double x = pts[3 * p] - C[0], y = pts[3 * p + 1] - C[1], z = pts[3 * p + 2] - C[2];
      for (int c = 0; c < ncart(l); c++, mu++) {
        int ea, eb, ec;
        cart_exponents(l, c, &ea, &eb, &ec);
        double v = 0, gx = 0, gy = 0, gz = 0, lap = 0;
        for (int q = 0; q < shell_nprim[s]; q++) {
          double al = alpha[prim + q], d = coef[prim + q];
          double px, px1, px2, py, py1, py2, pz, pz1, pz2;
          pow_d(x, ea, &px, &px1, &px2);
          pow_d(y, eb, &py, &py1, &py2);
          pow_d(z, ec, &pz, &pz1, &pz2);
          double ex = exp(-al * x * x), ey = exp(-al * y * y), ez = exp(-al * z * z);
          double X = px * ex, Y = py * ey, Zf = pz * ez;
          double X1 = (px1 - 2 * al * x * px) * ex;
          double Y1 = (py1 - 2 * al * y * py) * ey;
          double Z1 = (pz1 - 2 * al * z * pz) * ez;
          double X2 = (px2 - 2 * al * (2 * ea + 1) * px + 4 * al * al * x * x * px) * ex;
          double Y2 = (py2 - 2 * al * (2 * eb + 1) * py + 4 * al * al * y * y * py) * ey;
          double Z2 = (pz2 - 2 * al * (2 * ec + 1) * pz + 4 * al * al * z * z * pz) * ez;
          v += d * X * Y * Zf;
          gx += d * X1 * Y * Zf;
          gy += d * X * Y1 * Zf;
          gz += d * X * Y * Z1;
          lap += d * (X2 * Y * Zf + X * Y2 * Zf + X * Y * Z2);
        }
        o[0 * n_ao + mu] = v;
        o[1 * n_ao + mu] = gx;
        o[2 * n_ao + mu] = gy;
        o[3 * n_ao + mu] = gz;
        o[4 * n_ao + mu] = lap;
      }
      prim += shell_nprim[s];
    }
  }
  return 0;
}

/*
 * MO values and derivatives: phi_m = sum_mu B[mu][m] chi_mu for the value and
 * each of the four derivatives (linear in chi). mo_coef is n_ao x n_mo,
 * column-major (mo_coef[mu + n_ao*m]). out[p][0..4][m].
 */
int oracle_mo_eval(int n_shell, const int* shell_l, const int* shell_center,
                   const int* shell_nprim, const double* alpha, const double* coef,
                   const double* nuc_xyz, int n_mo, const double* mo_coef,
                   int n_pts, const double* pts, double* out) {
  int n_ao = oracle_n_ao(n_shell, shell_l);
  double* ao = (double*)malloc(sizeof(double) * 5 * n_ao);
  if (!ao) return -2;
  for (int p = 0; p < n_pts; p++) {
    int rc = oracle_ao_eval(n_shell, shell_l, shell_center, shell_nprim, alpha, coef,
                            nuc_xyz, 1, pts + 3 * p, ao);
    if (rc) { free(ao); return rc; }
    for (int c = 0; c < 5; c++)
      for (int m = 0; m < n_mo; m++) {
        nsum acc = {0, 0};
        for (int mu = 0; mu < n_ao; mu++) nadd(&acc, mo_coef[mu + (size_t)n_ao * m] * ao[c * n_ao + mu]);
        out[((size_t)p * 5 + c) * n_mo + m] = nval(&acc);
      }
  }
  free(ao);
  return 0;
}

/*
 * LU factorisation with partial pivoting (row interchanges), in place on a
 * row-major n x n matrix; piv[k] = row swapped with row k. Returns the number
 * of row interchanges, or -1 when a zero pivot is met (singular matrix).
 */
static int lu_pp(int n, double* a, int* piv) {
  int swaps = 0;
  for (int k = 0; k < n; k++) {
    int p = k;
    double best = fabs(a[k * n + k]);
    for (int i = k + 1; i < n; i++)
      if (fabs(a[i * n + k]) > best) { best = fabs(a[i * n + k]); p = i; }
    piv[k] = p;
    if (best == 0.0) return -1;
    if (p != k) {
      swaps++;
      for (int j = 0; j < n; j++) { double t = a[k * n + j]; a[k * n + j] = a[p * n + j]; a[p * n + j] = t; }
    }
    for (int i = k + 1; i < n; i++) {
      double f = a[i * n + k] / a[k * n + k];
      a[i * n + k] = f;
      for (int j = k + 1; j < n; j++) a[i * n + j] -= f * a[k * n + j];
    }
  }
  return swaps;
}

/* Determinant as (log|det|, sign) from an LU factorisation; sign 0 and
 * log = -inf for a singular matrix. a is row-major, left untouched. */
int oracle_det(int n, const double* a, double* logabs, int* sign) {
  if (n == 0) { *logabs = 0; *sign = 1; return 0; }
  double* w = (double*)malloc(sizeof(double) * n * n);
  int* piv = (int*)malloc(sizeof(int) * n);
  if (!w || !piv) { free(w); free(piv); return -2; }
  memcpy(w, a, sizeof(double) * n * n);
  int sw = lu_pp(n, w, piv);
  if (sw < 0) { *logabs = -INFINITY; *sign = 0; free(w); free(piv); return 0; }
  double la = 0; int sg = (sw & 1) ? -1 : 1;
  for (int k = 0; k < n; k++) { double d = w[k * n + k]; la += log(fabs(d)); if (d < 0) sg = -sg; }
  *logabs = la; *sign = sg;
  free(w); free(piv);
  return 0;
}

/* Inverse by LU solves of the unit columns; returns -1 if singular. */
int oracle_inverse(int n, const double* a, double* inv) {
  double* w = (double*)malloc(sizeof(double) * n * n);
  int* piv = (int*)malloc(sizeof(int) * n);
  double* col = (double*)malloc(sizeof(double) * n);
  if (!w || !piv || !col) { free(w); free(piv); free(col); return -2; }
  memcpy(w, a, sizeof(double) * n * n);
  if (lu_pp(n, w, piv) < 0) { free(w); free(piv); free(col); return -1; }
  for (int j = 0; j < n; j++) {
    for (int i = 0; i < n; i++) col[i] = (i == j) ? 1.0 : 0.0;
    for (int k = 0; k < n; k++) { double t = col[k]; col[k] = col[piv[k]]; col[piv[k]] = t; }
    for (int i = 0; i < n; i++) for (int k = 0; k < i; k++) col[i] -= w[i * n + k] * col[k];
    for (int i = n - 1; i >= 0; i--) {
      for (int k = i + 1; k < n; k++) col[i] -= w[i * n + k] * col[k];
      col[i] /= w[i * n + i];
    }
    for (int i = 0; i < n; i++) inv[i * n + j] = col[i];
  }
  free(w); free(piv); free(col);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Spin determinants                                                         */

/* Ascending list of occupied MOs (0-based) of a bit-string determinant:
 * bit (m mod 64) of word (m div 64) set <=> MO m occupied (Sec. 2.1). */
static int decode_occ(int n_int, const uint64_t* w, int* occ, int max_occ) {
  int n = 0;
  for (int q = 0; q < n_int; q++)
    for (int b = 0; b < 64; b++)
      if ((w[q] >> b) & 1ULL) { if (n < max_occ) occ[n] = 64 * q + b; n++; }
  return n;
}

/*
 * Value and derivatives of one spin determinant at one walker.
 * phi: [5][n_e_total][n_mo] MO table of the walker; e0: first electron of the
 * spin block; n: electrons of that spin; occ: ascending occupied MOs.
 * Outputs: log|D|, sign, and dD[i][mu] = (d_{i mu} D) / D  (i in the block,
 * mu = x, y, z, Laplacian) when D != 0. When D == 0 (singular Slater matrix)
 * the derivatives are returned unscaled in dD_abs (d_{i mu} D itself, computed
 * as determinants of the row-replaced matrices) and *sign = 0.
 * mode 0: cofactors from the inverse; mode 1: row-replaced determinants.
 */
static int spin_det(int n, int n_mo, int n_e, int e0, const double* phi, const int* occ,
                    int mode, double* logabs, int* sign, double* dD, double* dD_abs,
                    double* work /* >= 3 n^2 */) {
  double* S = work;
  double* inv = work + n * n;
  double* Sr = work + 2 * n * n;
  for (int i = 0; i < n; i++)
    for (int a = 0; a < n; a++) S[i * n + a] = phi[(0 * n_e + e0 + i) * n_mo + occ[a]];
  oracle_det(n, S, logabs, sign);
  int singular = (*sign == 0);
  if (!singular && mode == 0) {
    if (oracle_inverse(n, S, inv) != 0) singular = 1;
  }
  if (!singular && mode == 0) {
    for (int i = 0; i < n; i++)
      for (int mu = 0; mu < 4; mu++) {
        nsum acc = {0, 0};
        for (int a = 0; a < n; a++) nadd(&acc, phi[((1 + mu) * n_e + e0 + i) * n_mo + occ[a]] * inv[a * n + i]);
        dD[i * 4 + mu] = nval(&acc);
      }
    return 0;
  }
  /* row-replaced determinants: d_{i mu} D = Det(S with row i -> d_mu phi(r_i)) */
  for (int i = 0; i < n; i++)
    for (int mu = 0; mu < 4; mu++) {
      memcpy(Sr, S, sizeof(double) * n * n);
      for (int a = 0; a < n; a++) Sr[i * n + a] = phi[((1 + mu) * n_e + e0 + i) * n_mo + occ[a]];
      double la; int sg;
      oracle_det(n, Sr, &la, &sg);
      if (!singular) dD[i * 4 + mu] = sg * (*sign) * exp(la - *logabs);
      else dD_abs[i * 4 + mu] = sg * exp(la);
    }
  if (singular) *sign = 0;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Distinct spin determinants of the expansion (a generic sort; any order).  */
typedef struct { const uint64_t* w; int n_int; int64_t idx; } keyref;
static int cmp_keyref(const void* A, const void* B) {
  const keyref* a = (const keyref*)A; const keyref* b = (const keyref*)B;
  for (int q = a->n_int - 1; q >= 0; q--) {
    if (a->w[q] < b->w[q]) return -1;
    if (a->w[q] > b->w[q]) return 1;
  }
  return (a->idx < b->idx) ? -1 : (a->idx > b->idx);
}
/* map[k] = index of det k among the distinct ones; returns the count. */
static int64_t distinct_dets(int64_t n, int n_int, const uint64_t* dets, int64_t* map, int64_t* first) {
  keyref* r = (keyref*)malloc(sizeof(keyref) * (n ? n : 1));
  for (int64_t k = 0; k < n; k++) { r[k].w = dets + k * n_int; r[k].n_int = n_int; r[k].idx = k; }
  qsort(r, n, sizeof(keyref), cmp_keyref);
  int64_t u = -1;
  for (int64_t k = 0; k < n; k++) {
    if (k == 0 || memcmp(r[k].w, r[k - 1].w, sizeof(uint64_t) * n_int) != 0) { u++; first[u] = r[k].idx; }
    map[r[k].idx] = u;
  }
  free(r);
  return u + 1;
}

/* ------------------------------------------------------------------------ */
/* Full evaluation                                                           */
typedef struct {
  int n_up, n_dn, n_nuc; const double *Z, *nuc_xyz;
  int n_shell; const int *shell_l, *shell_center, *shell_nprim; const double *alpha, *coef;
  int n_mo; const double* mo_coef;
  int64_t n_det; int n_int; const uint64_t *det_up, *det_dn; const double* ci;
  int64_t nu_up, nu_dn; const int64_t *map_up, *map_dn, *first_up, *first_dn;
  const double* R; int mode;
  double *log_abs_psi, *grad, *lap, *e_local, *kappa; int* sign;
  int64_t w_begin, w_end; int status;
} job_t;

static double potential(int n_e, const double* r, int n_nuc, const double* Z, const double* X) {
  nsum v = {0, 0};
  for (int i = 0; i < n_e; i++)
    for (int A = 0; A < n_nuc; A++) {
      double dx = r[3 * i] - X[3 * A], dy = r[3 * i + 1] - X[3 * A + 1], dz = r[3 * i + 2] - X[3 * A + 2];
      nadd(&v, -Z[A] / sqrt(dx * dx + dy * dy + dz * dz));
    }
  for (int i = 0; i < n_e; i++)
    for (int j = i + 1; j < n_e; j++) {
      double dx = r[3 * i] - r[3 * j], dy = r[3 * i + 1] - r[3 * j + 1], dz = r[3 * i + 2] - r[3 * j + 2];
      nadd(&v, 1.0 / sqrt(dx * dx + dy * dy + dz * dz));
    }
  for (int A = 0; A < n_nuc; A++)
    for (int B = A + 1; B < n_nuc; B++) {
      double dx = X[3 * A] - X[3 * B], dy = X[3 * A + 1] - X[3 * B + 1], dz = X[3 * A + 2] - X[3 * B + 2];
      nadd(&v, Z[A] * Z[B] / sqrt(dx * dx + dy * dy + dz * dz));
    }
  return nval(&v);
}

/* Potential energy of n_e electrons at r[n_e][3] and n_nuc point nuclei of
 * charges Z at X[n_nuc][3] (the V of E_L, Sec. 4), exported for its pins. */
double oracle_potential(int n_e, const double* r, int n_nuc, const double* Z, const double* X) {
  return potential(n_e, r, n_nuc, Z, X);
}

static void* eval_job(void* arg) {
  job_t* J = (job_t*)arg;
  const int nu = J->n_up, nd = J->n_dn, ne = nu + nd, M = J->n_mo;
  const int nmax = nu > nd ? nu : nd;
  double* phi = (double*)malloc(sizeof(double) * 5 * ne * M);
  double* work = (double*)malloc(sizeof(double) * 3 * (nmax * nmax + 1));
  int* occ = (int*)malloc(sizeof(int) * (nmax + 1));
  /* per distinct det: scaled value d = sign*exp(log|D| - Lmax) and dD/D */
  double* la_up = (double*)malloc(sizeof(double) * J->nu_up);
  double* la_dn = (double*)malloc(sizeof(double) * J->nu_dn);
  int* sg_up = (int*)malloc(sizeof(int) * J->nu_up);
  int* sg_dn = (int*)malloc(sizeof(int) * J->nu_dn);
  double* dd_up = (double*)malloc(sizeof(double) * J->nu_up * 4 * (nu ? nu : 1));
  double* dd_dn = (double*)malloc(sizeof(double) * J->nu_dn * 4 * (nd ? nd : 1));
  double* da_up = (double*)malloc(sizeof(double) * J->nu_up * 4 * (nu ? nu : 1));
  double* da_dn = (double*)malloc(sizeof(double) * J->nu_dn * 4 * (nd ? nd : 1));
  double* v_up = (double*)malloc(sizeof(double) * J->nu_up);
  double* v_dn = (double*)malloc(sizeof(double) * J->nu_dn);
  nsum* G = (nsum*)malloc(sizeof(nsum) * 4 * ne);
  if (!phi || !work || !occ || !la_up || !la_dn || !sg_up || !sg_dn || !dd_up || !dd_dn ||
      !da_up || !da_dn || !v_up || !v_dn || !G) { J->status = -2; goto done; }
  for (int64_t w = J->w_begin; w < J->w_end; w++) {
    const double* r = J->R + (size_t)w * ne * 3;
    if (oracle_mo_eval(J->n_shell, J->shell_l, J->shell_center, J->shell_nprim, J->alpha, J->coef,
                       J->nuc_xyz, M, J->mo_coef, ne, r, phi)) { J->status = -3; goto done; }
    /* phi is [p][c][m]; spin_det wants [c][p][m] */
    double* phiT = (double*)malloc(sizeof(double) * 5 * ne * M);
    for (int p = 0; p < ne; p++) for (int c = 0; c < 5; c++)
      memcpy(phiT + ((size_t)c * ne + p) * M, phi + ((size_t)p * 5 + c) * M, sizeof(double) * M);
    for (int s = 0; s < 2; s++) {
      int n = s ? nd : nu, e0 = s ? nu : 0;
      int64_t cnt = s ? J->nu_dn : J->nu_up;
      const int64_t* first = s ? J->first_dn : J->first_up;
      const uint64_t* dets = s ? J->det_dn : J->det_up;
      double* la = s ? la_dn : la_up; int* sg = s ? sg_dn : sg_up;
      double* dd = s ? dd_dn : dd_up; double* da = s ? da_dn : da_up;
      for (int64_t I = 0; I < cnt; I++) {
        decode_occ(J->n_int, dets + first[I] * J->n_int, occ, nmax);
        spin_det(n, M, ne, e0, phiT, occ, J->mode, &la[I], &sg[I], dd + I * 4 * n, da + I * 4 * n, work);
      }
    }
    free(phiT);
    /* common scale per spin: the largest log|D| among the distinct dets */
    double Lu = -INFINITY, Ld = -INFINITY;
    for (int64_t I = 0; I < J->nu_up; I++) if (sg_up[I] && la_up[I] > Lu) Lu = la_up[I];
    for (int64_t I = 0; I < J->nu_dn; I++) if (sg_dn[I] && la_dn[I] > Ld) Ld = la_dn[I];
    if (!isfinite(Lu)) Lu = 0;
    if (!isfinite(Ld)) Ld = 0;
    for (int64_t I = 0; I < J->nu_up; I++) v_up[I] = sg_up[I] ? sg_up[I] * exp(la_up[I] - Lu) : 0.0;
    for (int64_t I = 0; I < J->nu_dn; I++) v_dn[I] = sg_dn[I] ? sg_dn[I] * exp(la_dn[I] - Ld) : 0.0;
    /* Eq. 1 and Eqs. 5-7 summed over the product list */
    nsum psi = {0, 0}, absum = {0, 0};
    for (int q = 0; q < 4 * ne; q++) { G[q].s = 0; G[q].c = 0; }
    for (int64_t k = 0; k < J->n_det; k++) {
      int64_t I = J->map_up[k], Jd = J->map_dn[k];
      double c = J->ci[k], du = v_up[I], dn = v_dn[Jd];
      nadd(&psi, c * du * dn);
      nadd(&absum, fabs(c * du * dn));
      for (int i = 0; i < nu; i++)
        for (int mu = 0; mu < 4; mu++) {
          double g = sg_up[I] ? du * dd_up[(I * nu + i) * 4 + mu] : da_up[(I * nu + i) * 4 + mu] * exp(-Lu);
          nadd(&G[i * 4 + mu], c * g * dn);
        }
      for (int i = 0; i < nd; i++)
        for (int mu = 0; mu < 4; mu++) {
          double g = sg_dn[Jd] ? dn * dd_dn[(Jd * nd + i) * 4 + mu] : da_dn[(Jd * nd + i) * 4 + mu] * exp(-Ld);
          nadd(&G[(nu + i) * 4 + mu], c * du * g);
        }
    }
    double P = nval(&psi);
    J->log_abs_psi[w] = (P == 0.0) ? -INFINITY : log(fabs(P)) + Lu + Ld;
    J->sign[w] = (P > 0) - (P < 0);
    J->kappa[w] = (P == 0.0) ? INFINITY : nval(&absum) / fabs(P);
    double tl = 0;
    for (int i = 0; i < ne; i++) {
      for (int d = 0; d < 3; d++) J->grad[((size_t)w * ne + i) * 3 + d] = nval(&G[i * 4 + d]) / P;
      double L = nval(&G[i * 4 + 3]) / P;
      J->lap[(size_t)w * ne + i] = L;
      tl += L;
    }
    J->e_local[w] = -0.5 * tl + potential(ne, r, J->n_nuc, J->Z, J->nuc_xyz);
  }
done:
  free(phi); free(work); free(occ); free(la_up); free(la_dn); free(sg_up); free(sg_dn);
  free(dd_up); free(dd_dn); free(da_up); free(da_dn); free(v_up); free(v_dn); free(G);
  return NULL;
}

/*
 * Psi, grad Psi / Psi, Lap_i Psi / Psi and E_L for n_walk walkers.
 * R: [n_walk][n_up+n_dn][3], electrons 0..n_up-1 are spin up.
 * det_up/det_dn: [n_det][n_int] bit strings; ci: [n_det].
 * Outputs: log_abs_psi[w], sign[w] (-1, 0, +1), grad[w][i][3], lap[w][i],
 * e_local[w], kappa[w] = sum_k |c_k D_up D_dn| / |Psi| (conditioning of the sum).
 * mode: 0 = cofactor derivatives, 1 = row-replaced determinants.
 * Returns 0, or a negative code on a malformed input.
 */
int oracle_evaluate(int n_up, int n_dn, int n_nuc, const double* Z, const double* nuc_xyz,
                    int n_shell, const int* shell_l, const int* shell_center, const int* shell_nprim,
                    const double* alpha, const double* coef, int n_mo, const double* mo_coef,
                    int64_t n_det, int n_int, const uint64_t* det_up, const uint64_t* det_dn,
                    const double* ci, int64_t n_walk, const double* R, int mode, int n_threads,
                    double* log_abs_psi, int* sign, double* grad, double* lap, double* e_local,
                    double* kappa) {
  if (n_up < 0 || n_dn < 0 || n_det < 1 || n_threads < 1) return -1;
  int occ_tmp[4096];
  for (int64_t k = 0; k < n_det; k++) {
    if (decode_occ(n_int, det_up + k * n_int, occ_tmp, 4096) != n_up) return -4;
    if (decode_occ(n_int, det_dn + k * n_int, occ_tmp, 4096) != n_dn) return -4;
    for (int a = 0; a < n_dn; a++) if (occ_tmp[a] >= n_mo) return -4;
    decode_occ(n_int, det_up + k * n_int, occ_tmp, 4096);
    for (int a = 0; a < n_up; a++) if (occ_tmp[a] >= n_mo) return -4;
  }
  int64_t* map_up = (int64_t*)malloc(sizeof(int64_t) * n_det);
  int64_t* map_dn = (int64_t*)malloc(sizeof(int64_t) * n_det);
  int64_t* first_up = (int64_t*)malloc(sizeof(int64_t) * n_det);
  int64_t* first_dn = (int64_t*)malloc(sizeof(int64_t) * n_det);
  int64_t nuu = distinct_dets(n_det, n_int, det_up, map_up, first_up);
  int64_t nud = distinct_dets(n_det, n_int, det_dn, map_dn, first_dn);
  if (n_threads > n_walk) n_threads = (int)(n_walk > 0 ? n_walk : 1);
  job_t* jobs = (job_t*)calloc(n_threads, sizeof(job_t));
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * n_threads);
  int rc = 0;
  for (int t = 0; t < n_threads; t++) {
    job_t* J = &jobs[t];
    J->n_up = n_up; J->n_dn = n_dn; J->n_nuc = n_nuc; J->Z = Z; J->nuc_xyz = nuc_xyz;
    J->n_shell = n_shell; J->shell_l = shell_l; J->shell_center = shell_center;
    J->shell_nprim = shell_nprim; J->alpha = alpha; J->coef = coef; J->n_mo = n_mo; J->mo_coef = mo_coef;
    J->n_det = n_det; J->n_int = n_int; J->det_up = det_up; J->det_dn = det_dn; J->ci = ci;
    J->nu_up = nuu; J->nu_dn = nud; J->map_up = map_up; J->map_dn = map_dn;
    J->first_up = first_up; J->first_dn = first_dn; J->R = R; J->mode = mode;
    J->log_abs_psi = log_abs_psi; J->sign = sign; J->grad = grad; J->lap = lap;
    J->e_local = e_local; J->kappa = kappa;
    J->w_begin = n_walk * t / n_threads; J->w_end = n_walk * (t + 1) / n_threads;
    pthread_create(&th[t], NULL, eval_job, J);
  }
  for (int t = 0; t < n_threads; t++) { pthread_join(th[t], NULL); if (jobs[t].status) rc = jobs[t].status; }
  free(jobs); free(th); free(map_up); free(map_dn); free(first_up); free(first_dn);
  return rc;
}

/*
 * Values of a list of spin determinants at walkers: for each walker w and each
 * determinant I (bit strings [n_dets][n_int], all of spin s with n electrons
 * starting at electron e0), log|D_I|, sign and dD[i][mu] / D.
 * out_log: [n_walk][n_dets], out_sign: [n_walk][n_dets],
 * out_dd: [n_walk][n_dets][n][4] (NaN when D_I == 0).
 */
int oracle_spin_dets(int n_e, int e0, int n, int n_shell, const int* shell_l, const int* shell_center,
                     const int* shell_nprim, const double* alpha, const double* coef,
                     const double* nuc_xyz, int n_mo, const double* mo_coef,
                     int64_t n_dets, int n_int, const uint64_t* dets, int64_t n_walk, const double* R,
                     int mode, double* out_log, int* out_sign, double* out_dd) {
  double* phi = (double*)malloc(sizeof(double) * 5 * n_e * n_mo);
  double* phiT = (double*)malloc(sizeof(double) * 5 * n_e * n_mo);
  double* work = (double*)malloc(sizeof(double) * 3 * (n * n + 1));
  double* da = (double*)malloc(sizeof(double) * 4 * (n + 1));
  int* occ = (int*)malloc(sizeof(int) * (n + 1));
  int rc = 0;
  for (int64_t w = 0; w < n_walk && !rc; w++) {
    rc = oracle_mo_eval(n_shell, shell_l, shell_center, shell_nprim, alpha, coef, nuc_xyz, n_mo,
                        mo_coef, n_e, R + (size_t)w * n_e * 3, phi);
    for (int p = 0; p < n_e; p++) for (int c = 0; c < 5; c++)
      memcpy(phiT + ((size_t)c * n_e + p) * n_mo, phi + ((size_t)p * 5 + c) * n_mo, sizeof(double) * n_mo);
    for (int64_t I = 0; I < n_dets && !rc; I++) {
      if (decode_occ(n_int, dets + I * n_int, occ, n) != n) { rc = -4; break; }
      double* dd = out_dd + ((size_t)w * n_dets + I) * n * 4;
      int sg;
      spin_det(n, n_mo, n_e, e0, phiT, occ, mode, &out_log[w * n_dets + I], &sg, dd, da, work);
      out_sign[w * n_dets + I] = sg;
      if (sg == 0) for (int q = 0; q < 4 * n; q++) dd[q] = NAN;
    }
  }
  free(phi); free(phiT); free(work); free(da); free(occ);
  return rc;
}
