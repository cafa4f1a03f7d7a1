/*
 * dqmc_oracle.c -- plain FP64 CPU oracle for the BSS/DQMC sweep of the ALF 1.0
 * documentation (Assaad et al., arXiv:1704.00131).
 *
 * TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and the CPU
 * baseline legs of bench.py load this library.  It shares no code, header or
 * table with the CUDA path of paper_1704_00131_gb300 and is never called by it.
 *
 * Everything is row-major double precision, written to be read against the
 * paper rather than to be fast: naive triple-loop products, cyclic Jacobi for
 * the symmetric eigenproblem, LU with partial pivoting, Householder QR with
 * column pivoting.  Each routine names the passage it follows.
 *
 * Notation (Sec. 2.1, Eqs. of the partition function and of G):
 *   N        lattice sites, L Trotter slices, beta = L * dtau
 *   K^s      hopping matrix of flavor s (includes -mu on the diagonal)
 *   E^s      = exp(-dtau K^s)                       (Op_T with g = -dtau)
 *   v^s_i,t  = sigma^s_k * c(field_k,t), site i = site(k)
 *   B^s_t    = E^s exp(V^s_t)                        (one-slice propagator)
 *   B(t2,t1) = B_t2 ... B_t1+1
 *   G^s(t)   = (1 + B^s(t,0) B^s(beta,t))^-1          (equal-time Green function)
 */
#include <complex.h>
#undef I /* the imaginary unit is written _Complex_I; I names a local below */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ESING 2

#define FIELD_ISING 1
#define FIELD_HS4 2

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11 "Parallel random numbers: */
/* as easy as 1, 2, 3"): 10 rounds of the 4x32 S-box with key schedule.      */
/* ------------------------------------------------------------------------ */
static void philox_round(uint32_t x[4], const uint32_t k[2]) {
  const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x[0];
  const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x[2];
  const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
  const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
  const uint32_t y0 = hi1 ^ x[1] ^ k[0];
  const uint32_t y1 = lo1;
  const uint32_t y2 = hi0 ^ x[3] ^ k[1];
  const uint32_t y3 = lo0;
  x[0] = y0; x[1] = y1; x[2] = y2; x[3] = y3;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t x[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
  uint32_t k[2] = {key[0], key[1]};
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k[0] += 0x9E3779B9u; k[1] += 0xBB67AE85u; }
    philox_round(x, k);
  }
  out[0] = x[0]; out[1] = x[1]; out[2] = x[2]; out[3] = x[3];
}

/* 53-bit uniform in [0,1) from two 32-bit words (high word first). */
double orc_u01(uint32_t hi, uint32_t lo) {
  const uint64_t w = ((uint64_t)hi << 32) | (uint64_t)lo;
  return (double)(w >> 11) * (1.0 / 9007199254740992.0);
}

/* The random words of one proposal: counter (sweep_lo, 2*tau+dir, k, sweep_hi),
 * key (seed_lo, seed_hi ^ chain).  u1 drives the proposal, u2 the acceptance. */
static void proposal_uniforms(uint64_t seed, uint32_t chain, uint64_t sweep, int tau,
                              int dir, int k, double* u1, double* u2) {
  uint32_t ctr[4] = {(uint32_t)sweep, (uint32_t)(2 * tau + dir), (uint32_t)k,
                     (uint32_t)(sweep >> 32)};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32) ^ chain};
  uint32_t o[4];
  orc_philox4x32_10(ctr, key, o);
  *u1 = orc_u01(o[0], o[1]);
  *u2 = orc_u01(o[2], o[3]);
}

/* Initial fields: counter domain (0xFFFFFFFF, tau, k, 0xFFFFFFFF).  Ising: -1 if
 * u1 < 1/2 else +1.  HS4: l = (-2,-1,1,2)[floor(4 u1)]. */
void orc_init_fields(int field_type, int L, int MV, uint64_t seed, uint32_t chain,
                     int8_t* fields /*[L][MV]*/) {
  static const int8_t hs4[4] = {-2, -1, 1, 2};
  for (int t = 0; t < L; ++t)
    for (int k = 0; k < MV; ++k) {
      uint32_t ctr[4] = {0xFFFFFFFFu, (uint32_t)(t + 1), (uint32_t)k, 0xFFFFFFFFu};
      uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32) ^ chain};
      uint32_t o[4];
      orc_philox4x32_10(ctr, key, o);
      const double u = orc_u01(o[0], o[1]);
      if (field_type == FIELD_ISING)
        fields[t * MV + k] = (u < 0.5) ? -1 : 1;
      else {
        int idx = (int)floor(4.0 * u);
        if (idx > 3) idx = 3;
        fields[t * MV + k] = hs4[idx];
      }
    }
}

/* ------------------------------------------------------------------------ */
/* Field couplings.                                                           */
/*  Ising (type 1, the Ising-coupled term exp(-dtau s I) of the partition     */
/*  function): exact two-valued decoupling of exp(-dtau U (n_up-1/2)(n_dn-1/2))*/
/*  with cosh(lambda) = exp(dtau U / 2); c(s) = lambda * s, weight 1.          */
/*  HS4 (type 2, the four-valued transform of Sec. 2.1 with M_z couplings     */
/*  g = sqrt(dtau U / 2), Sec. 6.2): c(l) = g * eta(l), weight gamma(l).       */
/* ------------------------------------------------------------------------ */
static double hs_eta(int l) {
  const double s6 = sqrt(6.0);
  switch (l) {
    case 1: return sqrt(2.0 * (3.0 - s6));
    case -1: return -sqrt(2.0 * (3.0 - s6));
    case 2: return sqrt(2.0 * (3.0 + s6));
    case -2: return -sqrt(2.0 * (3.0 + s6));
  }
  return NAN;
}
static double hs_gamma(int l) {
  const double s6 = sqrt(6.0);
  if (l == 1 || l == -1) return 1.0 + s6 / 3.0;
  if (l == 2 || l == -2) return 1.0 - s6 / 3.0;
  return NAN;
}

double orc_ising_lambda(double dtau, double U) { return acosh(exp(0.5 * dtau * U)); }

double orc_field_coupling(int field_type, double dtau, double U, int f) {
  if (field_type == FIELD_ISING) return orc_ising_lambda(dtau, U) * (double)f;
  return sqrt(0.5 * dtau * U) * hs_eta(f);
}

double orc_field_gamma(int field_type, int f) {
  if (field_type == FIELD_ISING) return 1.0;
  return hs_gamma(f);
}

/* d c(f) / dU */
static double field_coupling_dU(int field_type, double dtau, double U, int f) {
  if (field_type == FIELD_ISING) {
    const double lam = orc_ising_lambda(dtau, U);
    return 0.5 * dtau * exp(0.5 * dtau * U) / sinh(lam) * (double)f;
  }
  return dtau / (4.0 * sqrt(0.5 * dtau * U)) * hs_eta(f);
}

/* ------------------------------------------------------------------------ */
/* Dense linear algebra (row-major n x n).                                    */
/* ------------------------------------------------------------------------ */
static double* dalloc(size_t n) { return (double*)calloc(n ? n : 1, sizeof(double)); }

static void mat_mul(int n, const double* A, const double* B, double* C) {
  double* tmp = dalloc((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int k = 0; k < n; ++k) s += A[i * n + k] * B[k * n + j];
      tmp[i * n + j] = s;
    }
  memcpy(C, tmp, sizeof(double) * n * n);
  free(tmp);
}

static void mat_transpose(int n, const double* A, double* At) {
  double* tmp = dalloc((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) tmp[j * n + i] = A[i * n + j];
  memcpy(At, tmp, sizeof(double) * n * n);
  free(tmp);
}

static void mat_identity(int n, double* A) {
  memset(A, 0, sizeof(double) * n * n);
  for (int i = 0; i < n; ++i) A[i * n + i] = 1.0;
}

/* Symmetric eigendecomposition A = V diag(w) V^T by the cyclic Jacobi method
 * (Golub & Van Loan, Sec. 8.5).  Used for Op_set's exponentials (Table of the
 * Operator type: eigenvalues E and unitary U). */
int orc_eig_sym(int n, const double* A_in, double* w, double* V) {
  double* A = dalloc((size_t)n * n);
  memcpy(A, A_in, sizeof(double) * n * n);
  mat_identity(n, V);
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += A[p * n + q] * A[p * n + q];
    if (off < 1e-300) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[p * n + q];
        if (fabs(apq) < 1e-300) continue;
        const double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  /* columns p,q of A */
          const double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  /* rows p,q of A */
          const double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = c * vkp - s * vkq;
          V[k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  for (int i = 0; i < n; ++i) w[i] = A[i * n + i];
  free(A);
  return ORC_OK;
}

/* E = exp(t K) for symmetric K through K = V diag(w) V^T (Op_set). */
int orc_expm_sym(int n, const double* K, double t, double* E) {
  double* w = dalloc(n);
  double* V = dalloc((size_t)n * n);
  orc_eig_sym(n, K, w, V);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int k = 0; k < n; ++k) s += V[i * n + k] * exp(t * w[k]) * V[j * n + k];
      E[i * n + j] = s;
    }
  free(w);
  free(V);
  return ORC_OK;
}

/* LU with partial pivoting, in place.  Returns log|det| and sign; piv[n]. */
static int lu_factor(int n, double* A, int* piv, double* logdet, int* sign) {
  double ld = 0.0;
  int sg = 1;
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = fabs(A[k * n + k]);
    for (int i = k + 1; i < n; ++i)
      if (fabs(A[i * n + k]) > best) { best = fabs(A[i * n + k]); p = i; }
    piv[k] = p;
    if (best == 0.0) return ORC_ESING;
    if (p != k) {
      for (int j = 0; j < n; ++j) {
        const double t = A[k * n + j];
        A[k * n + j] = A[p * n + j];
        A[p * n + j] = t;
      }
      sg = -sg;
    }
    const double d = A[k * n + k];
    ld += log(fabs(d));
    if (d < 0) sg = -sg;
    for (int i = k + 1; i < n; ++i) {
      const double l = A[i * n + k] / d;
      A[i * n + k] = l;
      for (int j = k + 1; j < n; ++j) A[i * n + j] -= l * A[k * n + j];
    }
  }
  *logdet = ld;
  *sign = sg;
  return ORC_OK;
}

/* Solve (LU) X = B for n right-hand sides stored as the columns of B (in place). */
static void lu_solve(int n, const double* LU, const int* piv, double* B) {
  for (int k = 0; k < n; ++k)
    if (piv[k] != k)
      for (int j = 0; j < n; ++j) {
        const double t = B[k * n + j];
        B[k * n + j] = B[piv[k] * n + j];
        B[piv[k] * n + j] = t;
      }
  for (int j = 0; j < n; ++j) {
    for (int i = 0; i < n; ++i) {
      double s = B[i * n + j];
      for (int k = 0; k < i; ++k) s -= LU[i * n + k] * B[k * n + j];
      B[i * n + j] = s;
    }
    for (int i = n - 1; i >= 0; --i) {
      double s = B[i * n + j];
      for (int k = i + 1; k < n; ++k) s -= LU[i * n + k] * B[k * n + j];
      B[i * n + j] = s / LU[i * n + i];
    }
  }
}

/* log|det A| and sign by LU (brute force, used by tests for determinant ratios). */
int orc_logdet(int n, const double* A_in, double* logdet, int* sign) {
  double* A = dalloc((size_t)n * n);
  int* piv = (int*)calloc(n ? n : 1, sizeof(int));
  memcpy(A, A_in, sizeof(double) * n * n);
  int st = lu_factor(n, A, piv, logdet, sign);
  free(A);
  free(piv);
  return st;
}

/* Householder QR with column pivoting (Businger-Golub): A P = Q R.
 * Pivot: the remaining column of largest 2-norm, ties to the lowest index.
 * Q is formed explicitly (n x n), R is returned in A's upper triangle,
 * perm[k] = original column placed at position k, detQ = (-1)^reflections.
 * This is the "QR with pivoting" default of the stabilisation (Sec. 2.3). */
static void qr_pivoted(int n, double* A, double* Q, int* perm, int* detQ) {
  double* vs = dalloc((size_t)n * n); /* Householder vectors, row k = v_k */
  double* betas = dalloc(n);
  int dq = 1;
  for (int j = 0; j < n; ++j) perm[j] = j;
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = -1.0;
    for (int j = k; j < n; ++j) {
      double s = 0.0;
      for (int i = k; i < n; ++i) s += A[i * n + j] * A[i * n + j];
      if (s > best) { best = s; p = j; }
    }
    if (p != k) {
      for (int i = 0; i < n; ++i) {
        const double t = A[i * n + k];
        A[i * n + k] = A[i * n + p];
        A[i * n + p] = t;
      }
      const int t = perm[k]; perm[k] = perm[p]; perm[p] = t;
    }
    double nrm = 0.0;
    for (int i = k; i < n; ++i) nrm += A[i * n + k] * A[i * n + k];
    nrm = sqrt(nrm);
    double* v = vs + (size_t)k * n;
    betas[k] = 0.0;
    if (nrm == 0.0) continue;
    const double x0 = A[k * n + k];
    const double alpha = (x0 >= 0.0) ? -nrm : nrm;
    for (int i = 0; i < n; ++i) v[i] = 0.0;
    v[k] = x0 - alpha;
    for (int i = k + 1; i < n; ++i) v[i] = A[i * n + k];
    double vtv = 0.0;
    for (int i = k; i < n; ++i) vtv += v[i] * v[i];
    if (vtv == 0.0) continue;
    betas[k] = 2.0 / vtv;
    dq = -dq;
    for (int j = k; j < n; ++j) {
      double s = 0.0;
      for (int i = k; i < n; ++i) s += v[i] * A[i * n + j];
      s *= betas[k];
      for (int i = k; i < n; ++i) A[i * n + j] -= s * v[i];
    }
    A[k * n + k] = alpha;
    for (int i = k + 1; i < n; ++i) A[i * n + k] = 0.0;
  }
  /* Q = H_0 H_1 ... H_{n-1}, accumulated backwards onto the identity. */
  mat_identity(n, Q);
  for (int k = n - 1; k >= 0; --k) {
    if (betas[k] == 0.0) continue;
    const double* v = vs + (size_t)k * n;
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int i = k; i < n; ++i) s += v[i] * Q[i * n + j];
      s *= betas[k];
      for (int i = k; i < n; ++i) Q[i * n + j] -= s * v[i];
    }
  }
  *detQ = dq;
  free(vs);
  free(betas);
}

/* ------------------------------------------------------------------------ */
/* Model.                                                                     */
/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t n_sites, n_flavors, n_vertices, field_type, L, n_wrap;
  double dtau, U;
  const double* hopping;      /* [n_flavors][N][N] */
  const int32_t* vertex_site; /* [M_V] */
  const double* vertex_sign;  /* [n_flavors][M_V] */
} orc_model;

typedef struct {
  int N, nfl, MV, ft, L, nw;
  double dtau, U;
  double* K;     /* [nfl][N][N] */
  double* E;     /* exp(-dtau K) */
  double* Einv;  /* exp(+dtau K) */
  double* ET;    /* E^T */
  int* site;     /* [MV] */
  double* sgn;   /* [nfl][MV] */
} model_t;

static int model_load(const orc_model* m, model_t* M) {
  if (!m || m->n_sites <= 0 || m->n_flavors < 1 || m->n_flavors > 2 || m->n_vertices < 0 ||
      m->n_vertices > m->n_sites || m->L <= 0 || m->n_wrap <= 0 || m->L % m->n_wrap != 0 ||
      (m->field_type != FIELD_ISING && m->field_type != FIELD_HS4) || !(m->dtau > 0.0) ||
      m->U < 0.0)
    return ORC_EINVAL;
  const int N = m->n_sites;
  M->N = N; M->nfl = m->n_flavors; M->MV = m->n_vertices; M->ft = m->field_type;
  M->L = m->L; M->nw = m->n_wrap; M->dtau = m->dtau; M->U = m->U;
  const size_t nn = (size_t)N * N;
  M->K = dalloc(nn * M->nfl);
  M->E = dalloc(nn * M->nfl);
  M->Einv = dalloc(nn * M->nfl);
  M->ET = dalloc(nn * M->nfl);
  M->site = (int*)calloc(M->MV ? M->MV : 1, sizeof(int));
  M->sgn = dalloc((size_t)M->nfl * (M->MV ? M->MV : 1));
  memcpy(M->K, m->hopping, sizeof(double) * nn * M->nfl);
  for (int s = 0; s < M->nfl; ++s) {
    orc_expm_sym(N, M->K + s * nn, -M->dtau, M->E + s * nn);
    orc_expm_sym(N, M->K + s * nn, +M->dtau, M->Einv + s * nn);
    mat_transpose(N, M->E + s * nn, M->ET + s * nn);
  }
  for (int k = 0; k < M->MV; ++k) M->site[k] = m->vertex_site[k];
  for (int i = 0; i < M->nfl * M->MV; ++i) M->sgn[i] = m->vertex_sign[i];
  return ORC_OK;
}

static void model_free(model_t* M) {
  free(M->K); free(M->E); free(M->Einv); free(M->ET); free(M->site); free(M->sgn);
}

/* v^s at every site for slice tau (1-based), from fields [L][MV]. */
static void slice_potential(const model_t* M, const int8_t* fields, int s, int tau, double* v) {
  for (int i = 0; i < M->N; ++i) v[i] = 0.0;
  for (int k = 0; k < M->MV; ++k)
    v[M->site[k]] += M->sgn[s * M->MV + k] *
                     orc_field_coupling(M->ft, M->dtau, M->U, fields[(tau - 1) * M->MV + k]);
}

/* X <- B_tau X = E exp(V_tau) X */
static void apply_B_left(const model_t* M, const int8_t* f, int s, int tau, double* X) {
  const int N = M->N;
  double* v = dalloc(N);
  slice_potential(M, f, s, tau, v);
  for (int i = 0; i < N; ++i) {
    const double e = exp(v[i]);
    for (int j = 0; j < N; ++j) X[i * N + j] *= e;
  }
  mat_mul(N, M->E + (size_t)s * N * N, X, X);
  free(v);
}

/* X <- B_tau^T X = exp(V_tau) E^T X */
static void apply_BT_left(const model_t* M, const int8_t* f, int s, int tau, double* X) {
  const int N = M->N;
  double* v = dalloc(N);
  slice_potential(M, f, s, tau, v);
  mat_mul(N, M->ET + (size_t)s * N * N, X, X);
  for (int i = 0; i < N; ++i) {
    const double e = exp(v[i]);
    for (int j = 0; j < N; ++j) X[i * N + j] *= e;
  }
  free(v);
}

/* ------------------------------------------------------------------------ */
/* Exact result on fixed fields, by definition: G(tau) = (1 + B(tau,0)B(beta,tau))^-1 */
/* with the product formed plainly and the inverse by LU.  Valid while the    */
/* product is well conditioned (small beta * bandwidth).                      */
/* ------------------------------------------------------------------------ */
int orc_green_plain(const orc_model* m, const int8_t* fields, int s, int tau, double* G,
                    double* logdet, int* sign) {
  model_t M;
  int st = model_load(m, &M);
  if (st) return st;
  if (s < 0 || s >= M.nfl || tau < 0 || tau > M.L) { model_free(&M); return ORC_EINVAL; }
  const int N = M.N;
  double* A = dalloc((size_t)N * N);
  mat_identity(N, A);
  /* A = B(tau,0) B(beta,tau) = B_tau ... B_1 B_L ... B_tau+1: apply from the right end. */
  for (int t = tau + 1; t <= M.L; ++t) apply_B_left(&M, fields, s, t, A);
  for (int t = 1; t <= tau; ++t) apply_B_left(&M, fields, s, t, A);
  for (int i = 0; i < N; ++i) A[i * N + i] += 1.0;
  int* piv = (int*)calloc(N, sizeof(int));
  st = lu_factor(N, A, piv, logdet, sign);
  if (!st) {
    mat_identity(N, G);
    lu_solve(N, A, piv, G);
  }
  free(piv);
  free(A);
  model_free(&M);
  return st;
}

/* ------------------------------------------------------------------------ */
/* UDV chains (Sec. 2.3, Eq. green_stable and the three-step update):        */
/*   given A_{j-1} = Q D T,  M_j = (Bcal_j Q) D,  M_j P = Q' R,  D' = |diag R|, */
/*   T' = D'^-1 R P^T T.                                                       */
/* Right chain: B(tau,0) = Q_R D_R T_R.  Left chain: B(beta,tau)^T = Q_L D_L T_L. */
/* ------------------------------------------------------------------------ */
typedef struct { double *Q, *D, *T; int detQ; } udv_t;

static void udv_alloc(int N, udv_t* u) {
  u->Q = dalloc((size_t)N * N); u->D = dalloc(N); u->T = dalloc((size_t)N * N); u->detQ = 1;
}
static void udv_free(udv_t* u) { free(u->Q); free(u->D); free(u->T); }
static void udv_identity(int N, udv_t* u) {
  mat_identity(N, u->Q); mat_identity(N, u->T);
  for (int i = 0; i < N; ++i) u->D[i] = 1.0;
  u->detQ = 1;
}
static void udv_copy(int N, const udv_t* a, udv_t* b) {
  memcpy(b->Q, a->Q, sizeof(double) * N * N);
  memcpy(b->T, a->T, sizeof(double) * N * N);
  memcpy(b->D, a->D, sizeof(double) * N);
  b->detQ = a->detQ;
}

/* Given X = Bcal Q (already formed), finish the three steps in place on u. */
static void udv_finish(int N, double* X, udv_t* u) {
  /* M = X D (column scaling) */
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) X[i * N + j] *= u->D[j];
  int* perm = (int*)calloc(N, sizeof(int));
  double* Qn = dalloc((size_t)N * N);
  int dq;
  qr_pivoted(N, X, Qn, perm, &dq);
  /* D' = |diag R|;  T' = D'^-1 R P^T T  where (P^T T) row k = T row perm[k]. */
  double* Dn = dalloc(N);
  for (int k = 0; k < N; ++k) Dn[k] = fabs(X[k * N + k]);
  double* PT = dalloc((size_t)N * N);
  for (int k = 0; k < N; ++k) memcpy(PT + (size_t)k * N, u->T + (size_t)perm[k] * N, sizeof(double) * N);
  double* Tn = dalloc((size_t)N * N);
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) {
      double acc = 0.0;
      for (int k = i; k < N; ++k) acc += X[i * N + k] * PT[k * N + j];
      Tn[i * N + j] = (Dn[i] > 0.0) ? acc / Dn[i] : 0.0;
    }
  memcpy(u->Q, Qn, sizeof(double) * N * N);
  memcpy(u->T, Tn, sizeof(double) * N * N);
  memcpy(u->D, Dn, sizeof(double) * N);
  u->detQ = dq;
  free(perm); free(Qn); free(Dn); free(PT); free(Tn);
}

/* Right chain step: B(t1,0) -> B(t2,0) = B_t2 ... B_t1+1 B(t1,0). */
static void udv_right_step(const model_t* M, const int8_t* f, int s, int t1, int t2, udv_t* u) {
  const int N = M->N;
  double* X = dalloc((size_t)N * N);
  memcpy(X, u->Q, sizeof(double) * N * N);
  for (int t = t1 + 1; t <= t2; ++t) apply_B_left(M, f, s, t, X);
  udv_finish(N, X, u);
  free(X);
}

/* Left chain step: B(beta,t2)^T -> B(beta,t1)^T = B_t1+1^T ... B_t2^T B(beta,t2)^T. */
static void udv_left_step(const model_t* M, const int8_t* f, int s, int t1, int t2, udv_t* u) {
  const int N = M->N;
  double* X = dalloc((size_t)N * N);
  memcpy(X, u->Q, sizeof(double) * N * N);
  for (int t = t2; t >= t1 + 1; --t) apply_BT_left(M, f, s, t, X);
  udv_finish(N, X, u);
  free(X);
}

/* G = (1 + Q_R D_R T_R T_L^T D_L Q_L^T)^-1 by scale separation:
 *   D = Db * Ds, Db = max(D,1), Ds = min(D,1)
 *   Mid = Db_R^-1 Q_R^T Q_L Db_L^-1 + Ds_R (T_R T_L^T) Ds_L
 *   G   = Q_L Db_L^-1 Mid^-1 Db_R^-1 Q_R^T
 *   log|det G^-1| = sum log Db_R + sum log Db_L + log|det Mid|. */
static int green_from_udv(int N, const udv_t* R, const udv_t* Lf, double* G, double* logdet,
                          int* sign) {
  double* QRt = dalloc((size_t)N * N);
  double* QRtQL = dalloc((size_t)N * N);
  double* TLt = dalloc((size_t)N * N);
  double* TRTLt = dalloc((size_t)N * N);
  double* Mid = dalloc((size_t)N * N);
  double* X = dalloc((size_t)N * N);
  double *dbR = dalloc(N), *dsR = dalloc(N), *dbL = dalloc(N), *dsL = dalloc(N);
  for (int i = 0; i < N; ++i) {
    dbR[i] = R->D[i] > 1.0 ? R->D[i] : 1.0;
    dsR[i] = R->D[i] > 1.0 ? 1.0 : R->D[i];
    dbL[i] = Lf->D[i] > 1.0 ? Lf->D[i] : 1.0;
    dsL[i] = Lf->D[i] > 1.0 ? 1.0 : Lf->D[i];
  }
  mat_transpose(N, R->Q, QRt);
  mat_mul(N, QRt, Lf->Q, QRtQL);
  mat_transpose(N, Lf->T, TLt);
  mat_mul(N, R->T, TLt, TRTLt);
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j)
      Mid[i * N + j] = QRtQL[i * N + j] / (dbR[i] * dbL[j]) + dsR[i] * TRTLt[i * N + j] * dsL[j];
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) X[i * N + j] = QRt[i * N + j] / dbR[i];
  int* piv = (int*)calloc(N, sizeof(int));
  double ldm;
  int sm;
  int st = lu_factor(N, Mid, piv, &ldm, &sm);
  if (!st) {
    lu_solve(N, Mid, piv, X); /* X = Mid^-1 Db_R^-1 Q_R^T */
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < N; ++j) X[i * N + j] /= dbL[i];
    mat_mul(N, Lf->Q, X, G);
    double ld = ldm;
    for (int i = 0; i < N; ++i) ld += log(dbR[i]) + log(dbL[i]);
    *logdet = ld;
    *sign = sm * R->detQ * Lf->detQ;
  }
  free(piv); free(QRt); free(QRtQL); free(TLt); free(TRTLt); free(Mid); free(X);
  free(dbR); free(dsR); free(dbL); free(dsL);
  return st;
}

/* G(tau) from fixed fields through the two UDV chains, chunked every n_wrap
 * slices (right chain 0 -> tau, left chain beta -> tau); a partial chunk
 * closes each chain when tau is not a stabilisation point. */
int orc_green_udv(const orc_model* m, const int8_t* fields, int s, int tau, double* G,
                  double* logdet, int* sign) {
  model_t M;
  int st = model_load(m, &M);
  if (st) return st;
  if (s < 0 || s >= M.nfl || tau < 0 || tau > M.L) { model_free(&M); return ORC_EINVAL; }
  const int N = M.N, nw = M.nw;
  udv_t R, Lf;
  udv_alloc(N, &R); udv_alloc(N, &Lf);
  udv_identity(N, &R); udv_identity(N, &Lf);
  for (int t = 0; t < tau; t += nw) udv_right_step(&M, fields, s, t, (t + nw < tau) ? t + nw : tau, &R);
  for (int t = M.L; t > tau; t -= nw) udv_left_step(&M, fields, s, (t - nw > tau) ? t - nw : tau, t, &Lf);
  st = green_from_udv(N, &R, &Lf, G, logdet, sign);
  udv_free(&R); udv_free(&Lf);
  model_free(&M);
  return st;
}

/* ------------------------------------------------------------------------ */
/* Energy estimator (Sec. 6.1 observables, in the U n_up n_dn form):          */
/*   Kin  = sum_s sum_xy K^s_xy (delta_xy - G^s_yx)                          */
/*   Pot  = U sum_i (1 - G^up_ii)(1 - G^dn_ii)       (two flavors)           */
/*   Part = sum_s sum_i (1 - G^s_ii),   Ener = Kin + Pot.                    */
/* ------------------------------------------------------------------------ */
static void energy_terms(const model_t* M, double* const* G, double out[4]) {
  const int N = M->N;
  double kin = 0.0, pot = 0.0, part = 0.0;
  for (int s = 0; s < M->nfl; ++s) {
    const double* K = M->K + (size_t)s * N * N;
    for (int x = 0; x < N; ++x)
      for (int y = 0; y < N; ++y) kin += K[x * N + y] * ((x == y ? 1.0 : 0.0) - G[s][y * N + x]);
    for (int i = 0; i < N; ++i) part += 1.0 - G[s][i * N + i];
  }
  if (M->nfl == 2)
    for (int i = 0; i < N; ++i) pot += M->U * (1.0 - G[0][i * N + i]) * (1.0 - G[1][i * N + i]);
  out[0] = kin; out[1] = pot; out[2] = part; out[3] = kin + pot;
}

int orc_energy(const orc_model* m, const double* G_all /*[nfl][N][N]*/, double* out4) {
  model_t M;
  int st = model_load(m, &M);
  if (st) return st;
  double* G[2] = {(double*)G_all, (double*)G_all + (size_t)M.N * M.N * (M.nfl - 1)};
  energy_terms(&M, G, out4);
  model_free(&M);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* The Markov chain (Algorithm 1 with the default sequential single-field    */
/* updates of Sec. 2.2.1).                                                    */
/* ------------------------------------------------------------------------ */
typedef struct {
  int64_t proposals, accepted;
  double prec_green_mean, prec_green_max, prec_phase_max, mean_sign;
} orc_stats;

typedef struct {
  model_t M;
  uint64_t seed;
  uint32_t chain;
  uint64_t sweep;      /* sweeps done so far (Philox counter) */
  int8_t* fields;      /* [L][MV] */
  double* G[2];        /* current G (at tau = 0 between sweeps) */
  udv_t* slot[2];      /* [nst+1] per flavor */
  int sign;            /* sign of the current weight */
  int measure, meas_first, meas_last;
  double meas[4], sign_sum;
  int64_t n_meas;
  /* precision monitor of the last orc_chain_sweep call */
  double prec_sum, prec_max, phase_max;
  int64_t prec_events;
  int64_t proposals, accepted;
} orc_chain;

static void green_fresh(orc_chain* c, int s, int j_right, int j_left, double* G, double* ld,
                        int* sg) {
  /* j_right: slot index of the right chain (-1 = identity); j_left likewise. */
  const int N = c->M.N;
  udv_t I;
  udv_alloc(N, &I);
  udv_identity(N, &I);
  const udv_t* R = (j_right < 0) ? &I : &c->slot[s][j_right];
  const udv_t* Lf = (j_left < 0) ? &I : &c->slot[s][j_left];
  green_from_udv(N, R, Lf, G, ld, sg);
  udv_free(&I);
}

orc_chain* orc_chain_new(const orc_model* m, const int8_t* fields_or_null, uint64_t seed,
                         uint32_t chain, int measure, int meas_first, int meas_last) {
  orc_chain* c = (orc_chain*)calloc(1, sizeof(orc_chain));
  if (model_load(m, &c->M)) { free(c); return NULL; }
  const int N = c->M.N, L = c->M.L, MV = c->M.MV, nst = L / c->M.nw;
  c->seed = seed; c->chain = chain; c->sweep = 0;
  c->measure = measure; c->meas_first = meas_first; c->meas_last = meas_last;
  c->fields = (int8_t*)calloc((size_t)L * (MV ? MV : 1), 1);
  if (fields_or_null) memcpy(c->fields, fields_or_null, (size_t)L * MV);
  else orc_init_fields(c->M.ft, L, MV, seed, chain, c->fields);
  /* Fill the storage with the left chain (the wrapul loop of Algorithm 1). */
  c->sign = 1;
  for (int s = 0; s < c->M.nfl; ++s) {
    c->G[s] = dalloc((size_t)N * N);
    c->slot[s] = (udv_t*)calloc(nst + 1, sizeof(udv_t));
    for (int j = 0; j <= nst; ++j) udv_alloc(N, &c->slot[s][j]);
    udv_identity(N, &c->slot[s][nst]);
    for (int j = nst - 1; j >= 0; --j) {
      udv_copy(N, &c->slot[s][j + 1], &c->slot[s][j]);
      udv_left_step(&c->M, c->fields, s, j * c->M.nw, (j + 1) * c->M.nw, &c->slot[s][j]);
    }
    double ld;
    int sg;
    green_fresh(c, s, -1, 0, c->G[s], &ld, &sg);
    c->sign *= sg;
  }
  return c;
}

void orc_chain_free(orc_chain* c) {
  if (!c) return;
  const int nst = c->M.L / c->M.nw;
  for (int s = 0; s < c->M.nfl; ++s) {
    free(c->G[s]);
    for (int j = 0; j <= nst; ++j) udv_free(&c->slot[s][j]);
    free(c->slot[s]);
  }
  free(c->fields);
  model_free(&c->M);
  free(c);
}

/* G <- exp(a V_tau) G exp(-a V_tau), a = +1 (V-wrap) or -1 (V-unwrap). */
static void v_wrap(orc_chain* c, int s, int tau, double a) {
  const int N = c->M.N;
  double* v = dalloc(N);
  slice_potential(&c->M, c->fields, s, tau, v);
  for (int x = 0; x < N; ++x)
    for (int y = 0; y < N; ++y) c->G[s][x * N + y] *= exp(a * (v[x] - v[y]));
  free(v);
}

/* G <- X G Y (the hopping wrap: (E, E^-1) up, (E^-1, E) down). */
static void t_wrap(orc_chain* c, int s, int up) {
  const int N = c->M.N;
  const size_t nn = (size_t)N * N;
  if (up) {
    mat_mul(N, c->M.E + s * nn, c->G[s], c->G[s]);
    mat_mul(N, c->G[s], c->M.Einv + s * nn, c->G[s]);
  } else {
    mat_mul(N, c->M.Einv + s * nn, c->G[s], c->G[s]);
    mat_mul(N, c->G[s], c->M.E + s * nn, c->G[s]);
  }
}

/* One proposal at vertex k of slice tau (direction dir: 0 up, 1 down). */
static void propose(orc_chain* c, int tau, int dir, int k) {
  const model_t* M = &c->M;
  const int N = M->N, i = M->site[k];
  double u1, u2;
  proposal_uniforms(c->seed, c->chain, c->sweep, tau, dir, k, &u1, &u2);
  const int f = c->fields[(tau - 1) * M->MV + k];
  int fn;
  if (M->ft == FIELD_ISING) fn = -f;
  else {
    /* the three other values of (-2,-1,1,2), ascending, index floor(3 u1) */
    int others[3], n = 0;
    const int all[4] = {-2, -1, 1, 2};
    for (int q = 0; q < 4; ++q) if (all[q] != f) others[n++] = all[q];
    int idx = (int)floor(3.0 * u1);
    if (idx > 2) idx = 2;
    fn = others[idx];
  }
  const double dc = orc_field_coupling(M->ft, M->dtau, M->U, fn) -
                    orc_field_coupling(M->ft, M->dtau, M->U, f);
  double delta[2], Rs[2];
  double R = orc_field_gamma(M->ft, fn) / orc_field_gamma(M->ft, f);
  for (int s = 0; s < M->nfl; ++s) {
    delta[s] = exp(M->sgn[s * M->MV + k] * dc) - 1.0;
    Rs[s] = 1.0 + delta[s] * (1.0 - c->G[s][i * N + i]);
    R *= Rs[s];
  }
  c->proposals++;
  const double absR = fabs(R);
  if (u2 < (absR < 1.0 ? absR : 1.0)) {
    c->accepted++;
    c->fields[(tau - 1) * M->MV + k] = (int8_t)fn;
    if (R < 0) c->sign = -c->sign;
    /* Sherman-Morrison: G <- G - (delta/R_s) G[:,i] (e_i - G[i,:])^T */
    double* col = dalloc(N);
    double* row = dalloc(N);
    for (int s = 0; s < M->nfl; ++s) {
      double* G = c->G[s];
      const double fac = delta[s] / Rs[s];
      for (int x = 0; x < N; ++x) col[x] = G[x * N + i];
      for (int y = 0; y < N; ++y) row[y] = ((y == i) ? 1.0 : 0.0) - G[i * N + y];
      for (int x = 0; x < N; ++x)
        for (int y = 0; y < N; ++y) G[x * N + y] -= fac * col[x] * row[y];
    }
    free(col);
    free(row);
  }
}

/* One stabilisation event of flavor s (the cgr + control_precisionG steps of
 * Algorithm 1): G fresh from the right chain R and the left chain Lf replaces
 * the wrapped G; |G_wrap - G_fresh| feeds the precision monitor. */
static void fresh_replace(orc_chain* c, int s, const udv_t* R, const udv_t* Lf, int* fresh_sign) {
  const int N = c->M.N;
  double* Gf = dalloc((size_t)N * N);
  double ld, mx = 0.0, sm = 0.0;
  int sg = 1;
  green_from_udv(N, R, Lf, Gf, &ld, &sg);
  for (int x = 0; x < N * N; ++x) {
    const double d = fabs(Gf[x] - c->G[s][x]);
    sm += d;
    if (d > mx) mx = d;
  }
  memcpy(c->G[s], Gf, sizeof(double) * N * N);
  free(Gf);
  c->prec_sum += sm / ((double)N * N * c->M.nfl);
  if (mx > c->prec_max) c->prec_max = mx;
  *fresh_sign *= sg;
}

/* Close an event: the tracked sign is compared with the fresh one and replaced. */
static void close_event(orc_chain* c, int fresh_sign) {
  const double ph = fabs((double)fresh_sign - (double)c->sign);
  if (ph > c->phase_max) c->phase_max = ph;
  c->sign = fresh_sign;
  c->prec_events++;
}

static void measure_now(orc_chain* c, int tau) {
  if (!c->measure || tau < c->meas_first || tau > c->meas_last) return;
  double e[4];
  energy_terms(&c->M, c->G, e);
  for (int q = 0; q < 4; ++q) c->meas[q] += (double)c->sign * e[q];
  c->sign_sum += (double)c->sign;
  c->n_meas++;
}

/* One sweep: every field visited twice, tau = 1..L then L..1 (Sec. 2.4).
 * Upward slice tau:   V-wrap, proposals at vertices 0..MV-1, T-wrap to G(tau),
 *                     at tau = j*nw: right chain to tau, fresh G with the left
 *                     chain of slot j, slot j <- right chain.
 * Downward slice tau: T-unwrap, proposals at vertices MV-1..0, V-unwrap to
 *                     G(tau-1), at tau-1 = j*nw: left chain to tau-1, fresh G
 *                     with the right chain of slot j, slot j <- left chain. */
static void one_sweep(orc_chain* c) {
  const model_t* M = &c->M;
  const int N = M->N, L = M->L, nw = M->nw, nst = L / nw, nfl = M->nfl, MV = M->MV;
  udv_t chain, ident;
  udv_alloc(N, &chain);
  udv_alloc(N, &ident);
  udv_identity(N, &ident);
  for (int tau = 1; tau <= L; ++tau) {
    for (int s = 0; s < nfl; ++s) v_wrap(c, s, tau, +1.0);
    for (int k = 0; k < MV; ++k) propose(c, tau, 0, k);
    for (int s = 0; s < nfl; ++s) t_wrap(c, s, 1);
    if (tau % nw == 0) {
      const int j = tau / nw;
      int fs = 1;
      for (int s = 0; s < nfl; ++s) {
        udv_copy(N, (j == 1) ? &ident : &c->slot[s][j - 1], &chain);
        udv_right_step(M, c->fields, s, tau - nw, tau, &chain);
        fresh_replace(c, s, &chain, (j == nst) ? &ident : &c->slot[s][j], &fs);
        udv_copy(N, &chain, &c->slot[s][j]);
      }
      close_event(c, fs);
    }
    measure_now(c, tau);
  }
  for (int tau = L; tau >= 1; --tau) {
    for (int s = 0; s < nfl; ++s) t_wrap(c, s, 0);
    for (int k = MV - 1; k >= 0; --k) propose(c, tau, 1, k);
    for (int s = 0; s < nfl; ++s) v_wrap(c, s, tau, -1.0);
    const int t0 = tau - 1;
    if (t0 % nw == 0) {
      const int j = t0 / nw;
      int fs = 1;
      for (int s = 0; s < nfl; ++s) {
        udv_copy(N, (j + 1 == nst) ? &ident : &c->slot[s][j + 1], &chain);
        udv_left_step(M, c->fields, s, t0, t0 + nw, &chain);
        fresh_replace(c, s, (j == 0) ? &ident : &c->slot[s][j], &chain, &fs);
        udv_copy(N, &chain, &c->slot[s][j]);
      }
      close_event(c, fs);
    }
    measure_now(c, t0);
  }
  udv_free(&chain);
  udv_free(&ident);
  c->sweep++;
}

int orc_chain_sweep(orc_chain* c, int n_sweeps, orc_stats* st) {
  if (!c || n_sweeps < 0) return ORC_EINVAL;
  c->prec_sum = 0.0; c->prec_max = 0.0; c->phase_max = 0.0; c->prec_events = 0;
  c->proposals = 0; c->accepted = 0;
  double sgn_sum = 0.0;
  for (int n = 0; n < n_sweeps; ++n) {
    one_sweep(c);
    sgn_sum += (double)c->sign;
  }
  if (st) {
    st->proposals = c->proposals;
    st->accepted = c->accepted;
    st->prec_green_mean = c->prec_events ? c->prec_sum / (double)c->prec_events : 0.0;
    st->prec_green_max = c->prec_max;
    st->prec_phase_max = c->phase_max;
    st->mean_sign = n_sweeps ? sgn_sum / n_sweeps : 0.0;
  }
  return ORC_OK;
}

int orc_chain_green(const orc_chain* c, int s, double* G) {
  if (!c || s < 0 || s >= c->M.nfl) return ORC_EINVAL;
  memcpy(G, c->G[s], sizeof(double) * c->M.N * c->M.N);
  return ORC_OK;
}

int orc_chain_fields(const orc_chain* c, int8_t* out, uint64_t* sweep_counter, int* sign) {
  if (!c) return ORC_EINVAL;
  memcpy(out, c->fields, (size_t)c->M.L * c->M.MV);
  if (sweep_counter) *sweep_counter = c->sweep;
  if (sign) *sign = c->sign;
  return ORC_OK;
}

int orc_chain_measure(const orc_chain* c, double* out4, double* sign_sum, int64_t* n_meas) {
  if (!c) return ORC_EINVAL;
  for (int q = 0; q < 4; ++q) out4[q] = c->meas[q];
  *sign_sum = c->sign_sum;
  *n_meas = c->n_meas;
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Derivative of log|det(1 + B^s(beta,0))| on fixed fields.                  */
/* From G = (1 + B(beta,0))^-1 and d log det(1+B) = Tr[G dB]:                 */
/*   d log|det| = sum_tau Tr[(1 - G(tau-1)) B_tau^-1 dB_tau],                 */
/*   B_tau^-1 dB_tau = e^{-V} E^-1 dE e^{V} + dV,                            */
/* so with Gt_tau = e^{V_tau} G(tau-1) e^{-V_tau} and S = sum_tau (1 - Gt_tau): */
/*   hopping part: Tr[S E^-1 dE], dE the Frechet derivative of exp(-dtau K)  */
/*   in K's eigenbasis (Daleckii-Krein divided differences);                  */
/*   coupling part: sum_tau sum_k (1 - G(tau-1))_ii sigma_k dc(f_k,tau)/dU.    */
/* grad_K[s][x][y] = d/dK^s_xy with K_xy and K_yx varied together (x != y).   */
/* Each G(tau-1) is computed fresh through the UDV chains.                    */
/* ------------------------------------------------------------------------ */
int orc_logdet_grad(const orc_model* m, const int8_t* fields, double* logdet_out /*[nfl]*/,
                    int* sign_out /*[nfl]*/, double* grad_K /*[nfl][N][N]*/,
                    double* grad_U /*[nfl]*/) {
  model_t M;
  int st = model_load(m, &M);
  if (st) return st;
  const int N = M.N, L = M.L;
  const size_t nn = (size_t)N * N;
  double* G = dalloc(nn);
  double* S = dalloc(nn);
  double* v = dalloc(N);
  double* w = dalloc(N);
  double* V = dalloc(nn);
  double* A = dalloc(nn);
  double* Z = dalloc(nn);
  double* tmp = dalloc(nn);
  for (int s = 0; s < M.nfl; ++s) {
    memset(S, 0, sizeof(double) * nn);
    double gU = 0.0;
    for (int tau = 1; tau <= L; ++tau) {
      double ld;
      int sg;
      st = orc_green_udv(m, fields, s, tau - 1, G, &ld, &sg);
      if (st) goto done;
      if (tau == 1) { logdet_out[s] = ld; sign_out[s] = sg; }
      slice_potential(&M, fields, s, tau, v);
      for (int x = 0; x < N; ++x)
        for (int y = 0; y < N; ++y)
          S[x * N + y] += ((x == y) ? 1.0 : 0.0) - exp(v[x] - v[y]) * G[x * N + y];
      for (int k = 0; k < M.MV; ++k) {
        const int i = M.site[k];
        gU += (1.0 - G[i * N + i]) * M.sgn[s * M.MV + k] *
              field_coupling_dU(M.ft, M.dtau, M.U, fields[(tau - 1) * M.MV + k]);
      }
    }
    grad_U[s] = gU;
    /* A = S E^-1;  g = V [F o (V^T A^T V)] V^T;  F_ab divided differences of exp(-dtau x). */
    mat_mul(N, S, M.Einv + s * nn, A);
    orc_eig_sym(N, M.K + s * nn, w, V);
    mat_transpose(N, A, tmp);       /* A^T */
    mat_mul(N, tmp, V, Z);          /* A^T V */
    mat_transpose(N, V, tmp);       /* V^T */
    mat_mul(N, tmp, Z, Z);          /* V^T A^T V */
    for (int a = 0; a < N; ++a)
      for (int b = 0; b < N; ++b) {
        /* divided difference (e^{-t la} - e^{-t lb})/(la - lb), written without
         * cancellation: -t e^{-t(la+lb)/2} sinh(x)/x with x = t(la-lb)/2 */
        const double la = w[a], lb = w[b];
        const double x = 0.5 * M.dtau * (la - lb);
        const double shc = (x == 0.0) ? 1.0 : sinh(x) / x;
        Z[a * N + b] *= -M.dtau * exp(-0.5 * M.dtau * (la + lb)) * shc;
      }
    mat_mul(N, V, Z, Z);
    mat_mul(N, Z, tmp, Z);          /* V Z V^T */
    double* g = grad_K + s * nn;
    for (int x = 0; x < N; ++x)
      for (int y = 0; y < N; ++y) g[x * N + y] = (x == y) ? Z[x * N + y] : Z[x * N + y] + Z[y * N + x];
  }
done:
  free(G); free(S); free(v); free(w); free(V); free(A); free(Z); free(tmp);
  model_free(&M);
  return st;
}

/* ------------------------------------------------------------------------ */
/* Time-displaced Green functions on fixed fields (the equal-time G of Eq.   */
/* Green_eq extended to two times, Sec. 2.1 Observables):                    */
/*   G(tau,0) = B(tau,0) G(0) = (B(tau,0)^-1 + B(beta,tau))^-1                */
/*   G(0,tau) = -(1 - G(0)) B(tau,0)^-1 = -(B(tau,0) + B(beta,tau)^-1)^-1     */
/* From the two UDV chains, with the same middle matrix as the stable G:     */
/*   G(tau,0) = Q_L Db_L^-1 Mid^-1 Ds_R T_R                                   */
/*   G(0,tau) = -T_L^T Ds_L Mid^-1 Db_R^-1 Q_R^T                              */
/* ------------------------------------------------------------------------ */
static int displaced_from_udv(int N, const udv_t* R, const udv_t* Lf, double* Gt0, double* G0t) {
  double* QRt = dalloc((size_t)N * N);
  double* Mid = dalloc((size_t)N * N);
  double* TLt = dalloc((size_t)N * N);
  double* TT = dalloc((size_t)N * N);
  double* MI = dalloc((size_t)N * N);
  double* X = dalloc((size_t)N * N);
  mat_transpose(N, R->Q, QRt);
  mat_mul(N, QRt, Lf->Q, Mid);
  mat_transpose(N, Lf->T, TLt);
  mat_mul(N, R->T, TLt, TT);
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) {
      const double dR = R->D[i], dL = Lf->D[j];
      const double dbR = dR > 1.0 ? dR : 1.0, dsR = dR > 1.0 ? 1.0 : dR;
      const double dbL = dL > 1.0 ? dL : 1.0, dsL = dL > 1.0 ? 1.0 : dL;
      Mid[i * N + j] = Mid[i * N + j] / (dbR * dbL) + dsR * TT[i * N + j] * dsL;
    }
  int* piv = (int*)calloc(N, sizeof(int));
  double ld;
  int sg;
  int st = lu_factor(N, Mid, piv, &ld, &sg);
  if (!st) {
    mat_identity(N, MI);
    lu_solve(N, Mid, piv, MI); /* Mid^-1 */
    /* G(tau,0) = Q_L Db_L^-1 MI Ds_R T_R */
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < N; ++j) {
        const double dL = Lf->D[i];
        X[i * N + j] = MI[i * N + j] / (dL > 1.0 ? dL : 1.0);
      }
    mat_mul(N, Lf->Q, X, X);
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < N; ++j) {
        double acc = 0.0;
        for (int k = 0; k < N; ++k) {
          const double dR = R->D[k];
          acc += X[i * N + k] * (dR > 1.0 ? 1.0 : dR) * R->T[k * N + j];
        }
        Gt0[i * N + j] = acc;
      }
    /* G(0,tau) = -T_L^T Ds_L MI Db_R^-1 Q_R^T */
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < N; ++j) {
        const double dL = Lf->D[i];
        X[i * N + j] = (dL > 1.0 ? 1.0 : dL) * MI[i * N + j];
      }
    mat_mul(N, TLt, X, X);
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < N; ++j) {
        double acc = 0.0;
        for (int k = 0; k < N; ++k) {
          const double dR = R->D[k];
          acc += X[i * N + k] / (dR > 1.0 ? dR : 1.0) * QRt[k * N + j];
        }
        G0t[i * N + j] = -acc;
      }
  }
  free(QRt); free(Mid); free(TLt); free(TT); free(MI); free(X); free(piv);
  return st;
}

int orc_green_displaced(const orc_model* m, const int8_t* fields, int s, int tau, double* Gt0, double* G0t) {
  model_t M;
  int st = model_load(m, &M);
  if (st) return st;
  if (s < 0 || s >= M.nfl || tau < 0 || tau > M.L) { model_free(&M); return ORC_EINVAL; }
  const int N = M.N, nw = M.nw;
  udv_t R, Lf;
  udv_alloc(N, &R); udv_alloc(N, &Lf);
  udv_identity(N, &R); udv_identity(N, &Lf);
  for (int t = 0; t < tau; t += nw) udv_right_step(&M, fields, s, t, (t + nw < tau) ? t + nw : tau, &R);
  for (int t = M.L; t > tau; t -= nw) udv_left_step(&M, fields, s, (t - nw > tau) ? t - nw : tau, t, &Lf);
  st = displaced_from_udv(N, &R, &Lf, Gt0, G0t);
  udv_free(&R); udv_free(&Lf);
  model_free(&M);
  return st;
}

/* Derivative of the energy estimator E(G(0)) (the U n_up n_dn form above) on
 * fixed fields.  With Gamma^s = dE/dG^s = -(K^s)^T - diag(U (1 - G^sbar_ii)):
 *   dE = (explicit terms at fixed G) + sum_s Tr[Gamma^s^T dG^s],
 *   dG = -G dB(beta,0) G,  dB(beta,0) = sum_tau B(beta,tau) dB_tau B(tau-1,0),
 *   and B(tau-1,0) G = G(tau-1,0), G B(beta,tau) = -G(0,tau), so
 *   sum_s Tr[Gamma^T dG] = sum_s sum_tau Tr[Z_tau dB_tau],
 *   Z_tau = G(tau-1,0) Gamma^T G(0,tau),  dB_tau = dE e^{V} + E e^{V} dV.
 * Hopping part: Tr[e^{V} Z dE] through the Frechet derivative of exp(-dtau K)
 * (divided differences); coupling part: sum_i (Z E e^{V})_ii dv_i/dU.
 * energy_out = (Kin, Pot, Part, Ener) at G(0); grad_K[s] = dEner/dK^s with
 * K_xy and K_yx varied together (x != y); grad_U = dEner/dU. */
int orc_energy_grad(const orc_model* m, const int8_t* fields, double* energy_out, double* grad_K,
                    double* grad_U) {
  model_t M;
  int st = model_load(m, &M);
  if (st) return st;
  const int N = M.N, L = M.L, nfl = M.nfl;
  const size_t nn = (size_t)N * N;
  double* G0[2] = {dalloc(nn), dalloc(nn)};
  for (int s = 0; s < nfl; ++s) {
    double ld;
    int sg;
    st = orc_green_udv(m, fields, s, 0, G0[s], &ld, &sg);
    if (st) goto out;
  }
  energy_terms(&M, G0, energy_out);
  {
    double gu = 0.0;
    if (nfl == 2)
      for (int i = 0; i < N; ++i) gu += (1.0 - G0[0][i * N + i]) * (1.0 - G0[1][i * N + i]);
    double* Gam = dalloc(nn);
    double* Gt0 = dalloc(nn);
    double* G0t = dalloc(nn);
    double* Z = dalloc(nn);
    double* SE = dalloc(nn);
    double* T1 = dalloc(nn);
    double* v = dalloc(N);
    double* w = dalloc(N);
    double* V = dalloc(nn);
    for (int s = 0; s < nfl; ++s) {
      const double* K = M.K + s * nn;
      const double* E = M.E + s * nn;
      /* Gamma^T */
      for (int x = 0; x < N; ++x)
        for (int y = 0; y < N; ++y) {
          double g = -K[x * N + y]; /* (Gamma^T)_xy = Gamma_yx = -K_xy */
          if (x == y && nfl == 2) g -= M.U * (1.0 - G0[1 - s][x * N + x]);
          Gam[x * N + y] = g;
        }
      memset(SE, 0, sizeof(double) * nn);
      for (int tau = 1; tau <= L; ++tau) {
        st = orc_green_displaced(m, fields, s, tau - 1, Gt0, T1); /* G(tau-1,0); T1 unused */
        if (st) break;
        st = orc_green_displaced(m, fields, s, tau, T1, G0t);     /* G(0,tau);   T1 unused */
        if (st) break;
        mat_mul(N, Gt0, Gam, T1);  /* G(tau-1,0) Gamma^T */
        mat_mul(N, T1, G0t, Z);    /* Z_tau */
        slice_potential(&M, fields, s, tau, v);
        for (int x = 0; x < N; ++x)
          for (int y = 0; y < N; ++y) SE[x * N + y] += exp(v[x]) * Z[x * N + y];
        /* (Z E e^V)_ii dv_i/dU */
        for (int k = 0; k < M.MV; ++k) {
          const int i = M.site[k];
          double acc = 0.0;
          for (int q = 0; q < N; ++q) acc += Z[i * N + q] * E[q * N + i];
          acc *= exp(v[i]);
          gu += acc * M.sgn[s * M.MV + k] *
                field_coupling_dU(M.ft, M.dtau, M.U, fields[(tau - 1) * M.MV + k]);
        }
      }
      if (st) break;
      /* hopping: Tr[SE dE] -> V [F o (V^T SE^T V)] V^T, plus the explicit delta - G^T */
      orc_eig_sym(N, K, w, V);
      double* A = T1;
      mat_transpose(N, SE, A);         /* SE^T */
      mat_mul(N, A, V, Z);             /* SE^T V */
      mat_transpose(N, V, A);          /* V^T */
      mat_mul(N, A, Z, Z);             /* V^T SE^T V */
      for (int a = 0; a < N; ++a)
        for (int b = 0; b < N; ++b) {
          const double x = 0.5 * M.dtau * (w[a] - w[b]);
          const double shc = (x == 0.0) ? 1.0 : sinh(x) / x;
          Z[a * N + b] *= -M.dtau * exp(-0.5 * M.dtau * (w[a] + w[b])) * shc;
        }
      mat_mul(N, V, Z, Z);
      mat_mul(N, Z, A, Z);             /* V Z V^T: d/dK_xy of the implicit part */
      double* g = grad_K + s * nn;
      for (int x = 0; x < N; ++x)
        for (int y = 0; y < N; ++y) {
          /* explicit: d Kin / dK_xy = delta_xy - G_yx */
          const double ex = ((x == y) ? 1.0 : 0.0) - G0[s][y * N + x];
          const double exT = ((x == y) ? 1.0 : 0.0) - G0[s][x * N + y];
          if (x == y) g[x * N + y] = Z[x * N + y] + ex;
          else g[x * N + y] = Z[x * N + y] + Z[y * N + x] + ex + exT;
        }
    }
    *grad_U = gu;
    free(Gam); free(Gt0); free(G0t); free(Z); free(SE); free(T1); free(v); free(w); free(V);
  }
out:
  free(G0[0]); free(G0[1]);
  model_free(&M);
  return st;
}

/* Time-displaced measurement of one configuration (the tau_m step at the end
 * of a sweep, Algorithm 1; the ObserT quantities of Sec. 5.2): for each
 * displacement tau = 0..n_tau and flavor s, with G^s(tau,0), G^s(0,tau) and
 * G^s(tau,tau) each computed from scratch through the UDV chains,
 *   a_s(tau) = sum_x G^s(tau,0)_xx                        (local Green function)
 *   c_s(tau) = -sum_xy ph_x ph_y G^s(0,tau)_yx G^s(tau,0)_xy
 *              (Wick-connected part of sum_xy ph_x ph_y <n_xs(tau) n_ys(0)>)
 *   p_s(tau) = sum_x ph_x (1 - G^s(tau,tau)_xx)          (phase-weighted density)
 * out[(tau * nfl + s) * 3 + {0, 1, 2}] = (a_s, c_s, p_s); ph = NULL means 1.
 * sign_out[s] = sign of det(1 + B^s(beta,0)).
 * In one configuration the flavors are independent, so for two flavors
 *   sum_xy ph_x ph_y <S^z_x(tau) S^z_y(0)> =
 *     [(p_0(tau) - p_1(tau)) (p_0(0) - p_1(0)) + c_0(tau) + c_1(tau)] / 4. */
int orc_tau_observables(const orc_model* m, const int8_t* fields, int n_tau, const double* ph, double* out,
                        int* sign_out) {
  model_t M;
  int st = model_load(m, &M);
  if (st) return st;
  const int N = M.N, nfl = M.nfl;
  if (n_tau < 0 || n_tau > M.L) { model_free(&M); return ORC_EINVAL; }
  double* Gt0 = (double*)malloc(sizeof(double) * N * N);
  double* G0t = (double*)malloc(sizeof(double) * N * N);
  double* Gtt = (double*)malloc(sizeof(double) * N * N);
  for (int s = 0; s < nfl && !st; ++s) {
    for (int tau = 0; tau <= n_tau && !st; ++tau) {
      double ld;
      int sg;
      st = orc_green_displaced(m, fields, s, tau, Gt0, G0t);
      if (!st) st = orc_green_udv(m, fields, s, tau, Gtt, &ld, &sg);
      if (st) break;
      if (tau == 0) sign_out[s] = sg;
      double a = 0.0, c = 0.0, p = 0.0;
      for (int x = 0; x < N; ++x) {
        const double px = ph ? ph[x] : 1.0;
        a += Gt0[x * N + x];
        p += px * (1.0 - Gtt[x * N + x]);
        for (int y = 0; y < N; ++y) {
          const double py = ph ? ph[y] : 1.0;
          c -= px * py * G0t[y * N + x] * Gt0[x * N + y];
        }
      }
      double* o = out + ((size_t)tau * nfl + s) * 3;
      o[0] = a; o[1] = c; o[2] = p;
    }
  }
  free(Gt0); free(G0t); free(Gtt);
  model_free(&M);
  return st;
}

/* Time-displaced correlation functions per pair class of one configuration
 * (the ObserT quantities of Sec. 5.2 collected per lattice displacement, as
 * Obser_Latt does for the equal-time ones), spin-z decoupling with two flavors.
 * With G^s(tau,0)_xy = <c_xs(tau) c^+_ys(0)>, G^s(0,tau)_yx = -<c^+_xs(tau) c_ys(0)>,
 * m_x(tau) = sum_s sigma_s (1 - G^s(tau,tau)_xx), sigma = (+1, -1),
 * rho_x(tau) = sum_s (1 - G^s(tau,tau)_xx) and the Wick-connected
 * X^s_xy(tau) = -G^s(0,tau)_yx G^s(tau,0)_xy (flavors independent in one
 * configuration):
 *   sum_s <c_xs(tau) c^+_ys(0)>  = sum_s G^s(tau,0)_xy
 *   <S^z_x(tau) S^z_y(0)>        = [m_x(tau) m_y(0) + X^0_xy + X^1_xy] / 4
 *   <n_x(tau) n_y(0)>            = rho_x(tau) rho_y(0) + X^0_xy + X^1_xy
 * out[(tau * n_class + c) * 3 + {0, 1, 2}] = sums of these over the pairs
 * (x, y) with cls[x * N + y] == c, for tau = 0..n_tau; every Green function is
 * computed from scratch through the UDV chains.  At tau = 0 they reduce to the
 * equal-time G, S^z S^z and n n of orc_correlations. */
int orc_tau_correlations(const orc_model* m, const int8_t* fields, int n_tau, const int32_t* cls, int n_class,
                         double* out) {
  if (!m || m->n_flavors != 2 || n_class < 1 || n_tau < 0 || n_tau > m->L) return ORC_EINVAL;
  const int N = m->n_sites;
  for (int e = 0; e < N * N; ++e)
    if (cls[e] >= n_class) return ORC_EINVAL;
  const size_t NN = (size_t)N * N;
  double *Gt0[2], *G0t[2], *Gtt[2], *G00[2];
  for (int s = 0; s < 2; ++s) {
    Gt0[s] = dalloc(NN); G0t[s] = dalloc(NN); Gtt[s] = dalloc(NN); G00[s] = dalloc(NN);
  }
  int st = ORC_OK;
  double ld;
  int sg;
  for (int s = 0; s < 2 && !st; ++s) st = orc_green_udv(m, fields, s, 0, G00[s], &ld, &sg);
  for (int q = 0; q < (n_tau + 1) * n_class * 3; ++q) out[q] = 0.0;
  for (int tau = 0; tau <= n_tau && !st; ++tau) {
    for (int s = 0; s < 2 && !st; ++s) {
      st = orc_green_displaced(m, fields, s, tau, Gt0[s], G0t[s]);
      if (!st) st = orc_green_udv(m, fields, s, tau, Gtt[s], &ld, &sg);
    }
    if (st) break;
    for (int x = 0; x < N; ++x)
      for (int y = 0; y < N; ++y) {
        const int c = cls[x * N + y];
        if (c < 0) continue;
        const double nxu = 1.0 - Gtt[0][x * N + x], nxd = 1.0 - Gtt[1][x * N + x];
        const double nyu = 1.0 - G00[0][y * N + y], nyd = 1.0 - G00[1][y * N + y];
        const double X0 = -G0t[0][y * N + x] * Gt0[0][x * N + y];
        const double X1 = -G0t[1][y * N + x] * Gt0[1][x * N + y];
        double* o = out + ((size_t)tau * n_class + c) * 3;
        o[0] += Gt0[0][x * N + y] + Gt0[1][x * N + y];
        o[1] += 0.25 * ((nxu - nxd) * (nyu - nyd) + X0 + X1);
        o[2] += (nxu + nxd) * (nyu + nyd) + X0 + X1;
      }
  }
  for (int s = 0; s < 2; ++s) { free(Gt0[s]); free(G0t[s]); free(Gtt[s]); free(G00[s]); }
  return st;
}

/* Equal-time correlation functions of one configuration (the equal-time
 * observables of Sec. 5.2 and 6, Obser_Latt), for the spin-z decoupling with
 * two flavors (0 = up, 1 = down); G[s] is the equal-time Green function
 * G^s_xy = <c_xs c^+_ys> of the configuration.  Flavors are independent in one
 * configuration, so Wick's theorem gives, with rho_x = sum_s (1 - G^s_xx),
 * m_x = (1 - G^0_xx) - (1 - G^1_xx) and X^s_xy = (delta_xy - G^s_yx) G^s_xy:
 *   <S^z_x S^z_y> = [m_x m_y + X^0_xy + X^1_xy] / 4
 *   <n_x n_y>     = rho_x rho_y + X^0_xy + X^1_xy
 *   <S^+_x S^-_y> = (delta_xy - G^0_yx) G^1_xy
 *   sum_s <c^+_xs c_ys> = sum_s (delta_xy - G^s_yx)
 * out[c * 4 + {0, 1, 2, 3}] = sums of these over the pairs (x, y) with
 * cls[x * N + y] == c (0 <= c < n_class; pairs with a negative class skipped). */
int orc_correlations(int N, const double* G_all /*[2][N][N]*/, const int32_t* cls, int n_class, double* out) {
  if (N < 1 || n_class < 1) return ORC_EINVAL;
  const double* G0 = G_all;
  const double* G1 = G_all + (size_t)N * N;
  for (int q = 0; q < 4 * n_class; ++q) out[q] = 0.0;
  for (int x = 0; x < N; ++x)
    for (int y = 0; y < N; ++y) {
      const int c = cls[x * N + y];
      if (c < 0) continue;
      if (c >= n_class) return ORC_EINVAL;
      const double dxy = (x == y) ? 1.0 : 0.0;
      const double rx = (1.0 - G0[x * N + x]) + (1.0 - G1[x * N + x]);
      const double ry = (1.0 - G0[y * N + y]) + (1.0 - G1[y * N + y]);
      const double mx = (1.0 - G0[x * N + x]) - (1.0 - G1[x * N + x]);
      const double my = (1.0 - G0[y * N + y]) - (1.0 - G1[y * N + y]);
      const double X0 = (dxy - G0[y * N + x]) * G0[x * N + y];
      const double X1 = (dxy - G1[y * N + x]) * G1[x * N + y];
      out[c * 4 + 0] += 0.25 * (mx * my + X0 + X1);
      out[c * 4 + 1] += rx * ry + X0 + X1;
      out[c * 4 + 2] += (dxy - G0[y * N + x]) * G1[x * N + y];
      out[c * 4 + 3] += (dxy - G0[y * N + x]) + (dxy - G1[y * N + x]);
    }
  return ORC_OK;
}


/* ------------------------------------------------------------------------ */
/* SU(2) charge decoupling with complex coupling (the paper's default         */
/* Hubbard example, Sec. 6.1; the four-valued transform of Sec. 2.1 applied   */
/* to exp(-dtau U/2 (n_i - 1)^2), n_i = n_i,up + n_i,dn, whose quadratic form */
/* has the negative sign, hence the imaginary coupling):                      */
/*   exp(-dtau U/2 (n_i - 1)^2) = sum_l gamma(l)/4 exp(i g eta(l) (n_i - 1))   */
/*                                + O(dtau^4),   g = sqrt(dtau U / 2).        */
/* Both spins (colors) see the same one-body propagator, so on fixed fields   */
/*   B_tau = E exp(V_tau),  V_tau = diag(i g eta(l_tau,x)),  E = exp(-dtau K) */
/*   weight = prod gamma(l)/4 * exp(-i g sum eta(l)) * det(1 + B(beta,0))^2.  */
/* Plain product and complex LU with partial pivoting: valid for small        */
/* beta * bandwidth (no stabilisation).  TEST INFRASTRUCTURE (next row).      */
/* Outputs: G = (1 + B(beta,0))^-1 [N][N] complex (re, im interleaved),       */
/* log|det(1+B)|, arg det(1+B), the phase -g sum eta(l), and the energy       */
/* estimator per configuration (Wick, two colors):                            */
/*   Kin = 2 sum_xy K_xy (delta_xy - G_yx)                                     */
/*   Pot = U/2 sum_i <(n_i - 1)^2> = U/2 sum_i [2 (1-G_ii)^2 - 2 (1-G_ii) + 1] */
/* energy[0..3] = Re Kin, Im Kin, Re Pot, Im Pot.                              */
/* ------------------------------------------------------------------------ */
int orc_su2_plain(int N, const double* K, double dtau, double U, int L, const int8_t* fields, double* G_out,
                  double* logabs, double* arg, double* phase, double* energy) {
  if (N < 1 || L < 1 || !(dtau > 0.0) || !(U >= 0.0)) return ORC_EINVAL;
  for (int q = 0; q < L * N; ++q) {
    const int l = fields[q];
    if (l != 1 && l != -1 && l != 2 && l != -2) return ORC_EINVAL;
  }
  const size_t NN = (size_t)N * N;
  double* E = dalloc(NN);
  orc_expm_sym(N, K, -dtau, E);  /* exp(-dtau K) */
  double complex* B = (double complex*)calloc(NN, sizeof(double complex));
  double complex* T = (double complex*)calloc(NN, sizeof(double complex));
  for (int x = 0; x < N; ++x) B[(size_t)x * N + x] = 1.0;
  const double g = sqrt(0.5 * dtau * U);
  double ph = 0.0;
  /* B(beta,0) = B_L ... B_1: apply B_tau on the left for tau = 1..L */
  for (int tau = 1; tau <= L; ++tau) {
    for (int x = 0; x < N; ++x) {
      const double th = g * hs_eta(fields[(size_t)(tau - 1) * N + x]);
      ph -= th;
      const double complex ev = cexp(_Complex_I * th);
      for (int y = 0; y < N; ++y) B[(size_t)x * N + y] *= ev;
    }
    for (int x = 0; x < N; ++x)
      for (int y = 0; y < N; ++y) {
        double complex acc = 0.0;
        for (int k = 0; k < N; ++k) acc += E[(size_t)x * N + k] * B[(size_t)k * N + y];
        T[(size_t)x * N + y] = acc;
      }
    memcpy(B, T, NN * sizeof(double complex));
  }
  /* M = 1 + B; LU with partial pivoting; G = M^-1 column by column */
  for (int x = 0; x < N; ++x) B[(size_t)x * N + x] += 1.0;
  int* piv = (int*)malloc(sizeof(int) * N);
  double la = 0.0, ar = 0.0;
  int st = ORC_OK;
  for (int k = 0; k < N && !st; ++k) {
    int p = k;
    for (int i = k + 1; i < N; ++i)
      if (cabs(B[(size_t)i * N + k]) > cabs(B[(size_t)p * N + k])) p = i;
    piv[k] = p;
    if (cabs(B[(size_t)p * N + k]) == 0.0) { st = ORC_ESING; break; }
    if (p != k) {
      for (int j = 0; j < N; ++j) {
        const double complex t = B[(size_t)k * N + j];
        B[(size_t)k * N + j] = B[(size_t)p * N + j];
        B[(size_t)p * N + j] = t;
      }
      ar += 3.14159265358979323846;
    }
    const double complex d = B[(size_t)k * N + k];
    la += log(cabs(d));
    ar += carg(d);
    for (int i = k + 1; i < N; ++i) {
      const double complex l = B[(size_t)i * N + k] / d;
      B[(size_t)i * N + k] = l;
      for (int j = k + 1; j < N; ++j) B[(size_t)i * N + j] -= l * B[(size_t)k * N + j];
    }
  }
  if (!st) {
    double complex* col = (double complex*)malloc(sizeof(double complex) * N);
    double complex* G = (double complex*)malloc(sizeof(double complex) * NN);
    for (int j = 0; j < N; ++j) {
      for (int i = 0; i < N; ++i) col[i] = (i == j) ? 1.0 : 0.0;
      for (int k = 0; k < N; ++k) {
        const double complex t = col[k]; col[k] = col[piv[k]]; col[piv[k]] = t;
      }
      for (int i = 0; i < N; ++i)
        for (int k = 0; k < i; ++k) col[i] -= B[(size_t)i * N + k] * col[k];
      for (int i = N - 1; i >= 0; --i) {
        for (int k = i + 1; k < N; ++k) col[i] -= B[(size_t)i * N + k] * col[k];
        col[i] /= B[(size_t)i * N + i];
      }
      for (int i = 0; i < N; ++i) G[(size_t)i * N + j] = col[i];
    }
    double complex kin = 0.0, pot = 0.0;
    for (int x = 0; x < N; ++x)
      for (int y = 0; y < N; ++y) kin += 2.0 * K[(size_t)x * N + y] * ((x == y ? 1.0 : 0.0) - G[(size_t)y * N + x]);
    for (int i = 0; i < N; ++i) {
      const double complex h = 1.0 - G[(size_t)i * N + i];
      pot += 0.5 * U * (2.0 * h * h - 2.0 * h + 1.0);
    }
    for (size_t e = 0; e < NN; ++e) { G_out[2 * e] = creal(G[e]); G_out[2 * e + 1] = cimag(G[e]); }
    *logabs = la;
    *arg = remainder(ar, 2.0 * 3.14159265358979323846);
    *phase = ph;
    energy[0] = creal(kin); energy[1] = cimag(kin); energy[2] = creal(pot); energy[3] = cimag(pot);
    free(col); free(G);
  }
  free(piv); free(E); free(B); free(T);
  return st;
}

/* G~ = (1 + e^{V_tau} B(tau-1,0) B(beta,tau) E)^-1 of the SU(2) decoupling at
 * slice tau, from scratch (plain products): the Green function seen by the
 * vertices of slice tau, whose change multiplies B_tau = E e^{V_tau} on the
 * right of E.  Gt: [N][N] complex. */
static int su2_green_at_vertex(int N, const double* E, double g, int L, const int8_t* fields, int tau,
                               double complex* Gt) {
  const size_t NN = (size_t)N * N;
  double complex* A = (double complex*)calloc(NN, sizeof(double complex));
  double complex* T = (double complex*)calloc(NN, sizeof(double complex));
  for (int x = 0; x < N; ++x) A[(size_t)x * N + x] = 1.0;
  /* A <- E, then left-multiply B_L ... B_tau+1, then B_tau-1 ... B_1, then e^{V_tau} */
  for (int x = 0; x < N; ++x)
    for (int y = 0; y < N; ++y) A[(size_t)x * N + y] = E[(size_t)x * N + y];
  for (int step = 0; step < L - 1; ++step) {
    const int t = (tau + 1 + step - 1) % L + 1;   /* tau+1, ..., L, 1, ..., tau-1 */
    for (int x = 0; x < N; ++x) {
      const double complex ev = cexp(_Complex_I * g * hs_eta(fields[(size_t)(t - 1) * N + x]));
      for (int y = 0; y < N; ++y) A[(size_t)x * N + y] *= ev;
    }
    for (int x = 0; x < N; ++x)
      for (int y = 0; y < N; ++y) {
        double complex acc = 0.0;
        for (int k = 0; k < N; ++k) acc += E[(size_t)x * N + k] * A[(size_t)k * N + y];
        T[(size_t)x * N + y] = acc;
      }
    memcpy(A, T, NN * sizeof(double complex));
  }
  for (int x = 0; x < N; ++x) {
    const double complex ev = cexp(_Complex_I * g * hs_eta(fields[(size_t)(tau - 1) * N + x]));
    for (int y = 0; y < N; ++y) A[(size_t)x * N + y] *= ev;
  }
  /* Gt = (1 + A)^-1 by Gauss-Jordan with partial pivoting */
  for (int x = 0; x < N; ++x) A[(size_t)x * N + x] += 1.0;
  for (size_t e = 0; e < NN; ++e) Gt[e] = 0.0;
  for (int x = 0; x < N; ++x) Gt[(size_t)x * N + x] = 1.0;
  int st = ORC_OK;
  for (int k = 0; k < N; ++k) {
    int p = k;
    for (int i = k + 1; i < N; ++i)
      if (cabs(A[(size_t)i * N + k]) > cabs(A[(size_t)p * N + k])) p = i;
    if (cabs(A[(size_t)p * N + k]) == 0.0) { st = ORC_ESING; break; }
    for (int j = 0; j < N; ++j) {
      double complex t = A[(size_t)k * N + j]; A[(size_t)k * N + j] = A[(size_t)p * N + j]; A[(size_t)p * N + j] = t;
      t = Gt[(size_t)k * N + j]; Gt[(size_t)k * N + j] = Gt[(size_t)p * N + j]; Gt[(size_t)p * N + j] = t;
    }
    const double complex d = A[(size_t)k * N + k];
    for (int j = 0; j < N; ++j) { A[(size_t)k * N + j] /= d; Gt[(size_t)k * N + j] /= d; }
    for (int i = 0; i < N; ++i) {
      if (i == k) continue;
      const double complex f = A[(size_t)i * N + k];
      for (int j = 0; j < N; ++j) {
        A[(size_t)i * N + j] -= f * A[(size_t)k * N + j];
        Gt[(size_t)i * N + j] -= f * Gt[(size_t)k * N + j];
      }
    }
  }
  free(A); free(T);
  return st;
}

/* One sweep of a Markov chain of the SU(2) decoupling (the paper's sampling
 * with complex weights: W(C) = |Re e^{-S(C)}| (Sec. 2.2), Metropolis on W).
 * Order and random numbers as for the spin-z chains: up tau = 1..L with sites
 * 0..N-1, down tau = L..1 with sites N-1..0; Philox counter (sweep_lo, 2 tau +
 * dir, site, sweep_hi), key (seed_lo, seed_hi ^ chain); the proposal is one of
 * the other three field values (ascending, index floor(3 u1)).  Per proposal,
 * with Delta = e^{i g (eta' - eta)} - 1 and G~ from su2_green_at_vertex,
 *   R = gamma(l')/gamma(l) * e^{-i g (eta' - eta)} * (1 + Delta (1 - G~_ii))^2,
 * accepted when u2 < |Re(P R)| / |Re P|, P the phase of e^{-S(C)} (in/out as
 * phase[0] + i phase[1]; on entry with phase[0] = phase[1] = 0 it is computed).
 * After the sweep: energy estimator of the final configuration at tau = 0,
 * reweighted as in Sec. 2.2: obs[0..1] = sign * (P / Re P) * (Kin + Pot)
 * (re, im), obs[2] = sign.  accepted: number of accepted proposals. */
int orc_su2_sweep(int N, const double* K, double dtau, double U, int L, int8_t* fields, uint64_t seed,
                  uint32_t chain, uint64_t sweep, double* phase, double* obs, int* accepted) {
  if (N < 1 || L < 1 || !(dtau > 0.0) || !(U >= 0.0)) return ORC_EINVAL;
  const size_t NN = (size_t)N * N;
  const double g = sqrt(0.5 * dtau * U);
  double* E = dalloc(NN);
  orc_expm_sym(N, K, -dtau, E);
  double complex* Gt = (double complex*)malloc(NN * sizeof(double complex));
  double* Gd = dalloc(2 * NN);
  double la, ar, ph, en[4];
  int st = ORC_OK;
  double complex P = phase[0] + _Complex_I * phase[1];
  if (phase[0] == 0.0 && phase[1] == 0.0) {
    st = orc_su2_plain(N, K, dtau, U, L, fields, Gd, &la, &ar, &ph, en);
    if (st) { free(E); free(Gt); free(Gd); return st; }
    P = cexp(_Complex_I * (ph + 2.0 * ar));   /* prod gamma/4 > 0 and |det|^2 do not change the phase */
  }
  int acc = 0;
  for (int dir = 0; dir < 2 && !st; ++dir) {
    for (int step = 0; step < L && !st; ++step) {
      const int tau = dir ? L - step : step + 1;
      for (int q = 0; q < N; ++q) {
        const int k = dir ? N - 1 - q : q;
        double u1, u2;
        proposal_uniforms(seed, chain, sweep, tau, dir, k, &u1, &u2);
        const int f = fields[(size_t)(tau - 1) * N + k];
        int others[3], n = 0;
        const int all[4] = {-2, -1, 1, 2};
        for (int a = 0; a < 4; ++a) if (all[a] != f) others[n++] = all[a];
        int idx = (int)floor(3.0 * u1);
        if (idx > 2) idx = 2;
        const int fn = others[idx];
        st = su2_green_at_vertex(N, E, g, L, fields, tau, Gt);
        if (st) break;
        const double dth = g * (hs_eta(fn) - hs_eta(f));
        const double complex delta = cexp(_Complex_I * dth) - 1.0;
        const double complex r1 = 1.0 + delta * (1.0 - Gt[(size_t)k * N + k]);
        const double complex R = hs_gamma(fn) / hs_gamma(f) * cexp(-_Complex_I * dth) * r1 * r1;
        const double ratio = fabs(creal(P * R)) / fabs(creal(P));
        if (u2 < (ratio < 1.0 ? ratio : 1.0)) {
          fields[(size_t)(tau - 1) * N + k] = (int8_t)fn;
          P = P * R / cabs(P * R);
          ++acc;
        }
      }
    }
  }
  if (!st) st = orc_su2_plain(N, K, dtau, U, L, fields, Gd, &la, &ar, &ph, en);
  if (!st) {
    const double sgn = creal(P) >= 0.0 ? 1.0 : -1.0;
    const double complex w = sgn * P / creal(P) * ((en[0] + _Complex_I * en[1]) + (en[2] + _Complex_I * en[3]));
    obs[0] = creal(w); obs[1] = cimag(w); obs[2] = sgn;
    phase[0] = creal(P); phase[1] = cimag(P);
    *accepted = acc;
  }
  free(E); free(Gt); free(Gd);
  return st;
}

/* ---- complex UDV chain of the SU(2) decoupling (stable G at any beta) ----- */
/* The steps of the real chain with complex arithmetic: Householder reflectors */
/* H = 1 - 2 v v^H / (v^H v) (unitary, det -1), column pivoting on the norms,  */
/* D = |diag R|, T = D^-1 R P^T T.  The left chain stores B(beta,tau)^H, so    */
/*   1 + B(tau,0) B(beta,tau) = Q_R Db_R Mid Db_L Q_L^H,                        */
/*   Mid = Db_R^-1 Q_R^H Q_L Db_L^-1 + Ds_R T_R T_L^H Ds_L,                     */
/*   G = Q_L Db_L^-1 Mid^-1 Db_R^-1 Q_R^H,                                      */
/*   det(1 + B) = det Q_R conj(det Q_L) prod Db_R prod Db_L det Mid.            */
typedef struct { double complex *Q, *T; double* D; int detQ; } cudv_t;

static void cudv_alloc(int N, cudv_t* u) {
  u->Q = (double complex*)calloc((size_t)N * N, sizeof(double complex));
  u->T = (double complex*)calloc((size_t)N * N, sizeof(double complex));
  u->D = dalloc(N);
  for (int i = 0; i < N; ++i) { u->Q[(size_t)i * N + i] = 1.0; u->T[(size_t)i * N + i] = 1.0; u->D[i] = 1.0; }
  u->detQ = 1;
}
static void cudv_free(cudv_t* u) { free(u->Q); free(u->T); free(u->D); }

static void cudv_finish(int N, double complex* X, cudv_t* u) {
  const size_t NN = (size_t)N * N;
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) X[(size_t)i * N + j] *= u->D[j];
  int* perm = (int*)calloc(N, sizeof(int));
  double complex* vs = (double complex*)calloc(NN, sizeof(double complex));
  double* betas = dalloc(N);
  int dq = 1;
  for (int j = 0; j < N; ++j) perm[j] = j;
  for (int k = 0; k < N; ++k) {
    int p = k;
    double best = -1.0;
    for (int j = k; j < N; ++j) {
      double s = 0.0;
      for (int i = k; i < N; ++i) { const double a = cabs(X[(size_t)i * N + j]); s += a * a; }
      if (s > best) { best = s; p = j; }
    }
    if (p != k) {
      for (int i = 0; i < N; ++i) {
        const double complex t = X[(size_t)i * N + k]; X[(size_t)i * N + k] = X[(size_t)i * N + p]; X[(size_t)i * N + p] = t;
      }
      const int t = perm[k]; perm[k] = perm[p]; perm[p] = t;
    }
    double nrm = 0.0;
    for (int i = k; i < N; ++i) { const double a = cabs(X[(size_t)i * N + k]); nrm += a * a; }
    nrm = sqrt(nrm);
    betas[k] = 0.0;
    if (nrm == 0.0) continue;
    double complex* v = vs + (size_t)k * N;
    const double complex x0 = X[(size_t)k * N + k];
    const double complex alpha = (cabs(x0) > 0.0) ? -x0 / cabs(x0) * nrm : -nrm;
    v[k] = x0 - alpha;
    for (int i = k + 1; i < N; ++i) v[i] = X[(size_t)i * N + k];
    double vhv = 0.0;
    for (int i = k; i < N; ++i) { const double a = cabs(v[i]); vhv += a * a; }
    if (vhv == 0.0) continue;
    betas[k] = 2.0 / vhv;
    dq = -dq;
    for (int j = k; j < N; ++j) {
      double complex s = 0.0;
      for (int i = k; i < N; ++i) s += conj(v[i]) * X[(size_t)i * N + j];
      s *= betas[k];
      for (int i = k; i < N; ++i) X[(size_t)i * N + j] -= s * v[i];
    }
    X[(size_t)k * N + k] = alpha;
    for (int i = k + 1; i < N; ++i) X[(size_t)i * N + k] = 0.0;
  }
  /* Q = H_0 ... H_{N-1} applied to the identity from the last reflector */
  double complex* Qn = (double complex*)calloc(NN, sizeof(double complex));
  for (int i = 0; i < N; ++i) Qn[(size_t)i * N + i] = 1.0;
  for (int k = N - 1; k >= 0; --k) {
    if (betas[k] == 0.0) continue;
    const double complex* v = vs + (size_t)k * N;
    for (int j = 0; j < N; ++j) {
      double complex s = 0.0;
      for (int i = k; i < N; ++i) s += conj(v[i]) * Qn[(size_t)i * N + j];
      s *= betas[k];
      for (int i = k; i < N; ++i) Qn[(size_t)i * N + j] -= s * v[i];
    }
  }
  double* Dn = dalloc(N);
  for (int k = 0; k < N; ++k) Dn[k] = cabs(X[(size_t)k * N + k]);
  double complex* Tn = (double complex*)calloc(NN, sizeof(double complex));
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) {
      double complex acc = 0.0;
      for (int k = i; k < N; ++k) acc += X[(size_t)i * N + k] * u->T[(size_t)perm[k] * N + j];
      Tn[(size_t)i * N + j] = (Dn[i] > 0.0) ? acc / Dn[i] : 0.0;
    }
  memcpy(u->Q, Qn, NN * sizeof(double complex));
  memcpy(u->T, Tn, NN * sizeof(double complex));
  memcpy(u->D, Dn, (size_t)N * sizeof(double));
  u->detQ = dq;
  free(perm); free(vs); free(betas); free(Qn); free(Dn); free(Tn);
}

/* Right chain: X <- B_t X = E e^{i g eta} X for t = t1+1..t2.  Left chain:
 * X <- B_t^H X = e^{-i g eta} E X for t = t2..t1+1. */
static void cudv_step(int N, const double* E, double g, const int8_t* fields, int t1, int t2, int left,
                      cudv_t* u) {
  const size_t NN = (size_t)N * N;
  double complex* X = (double complex*)malloc(NN * sizeof(double complex));
  double complex* Y = (double complex*)malloc(NN * sizeof(double complex));
  memcpy(X, u->Q, NN * sizeof(double complex));
  for (int step = 0; step < t2 - t1; ++step) {
    const int t = left ? t2 - step : t1 + 1 + step;
    if (!left)
      for (int x = 0; x < N; ++x) {
        const double complex ev = cexp(_Complex_I * g * hs_eta(fields[(size_t)(t - 1) * N + x]));
        for (int y = 0; y < N; ++y) X[(size_t)x * N + y] *= ev;
      }
    for (int x = 0; x < N; ++x)
      for (int y = 0; y < N; ++y) {
        double complex acc = 0.0;
        for (int k = 0; k < N; ++k) acc += E[(size_t)x * N + k] * X[(size_t)k * N + y];
        Y[(size_t)x * N + y] = acc;
      }
    memcpy(X, Y, NN * sizeof(double complex));
    if (left)
      for (int x = 0; x < N; ++x) {
        const double complex ev = cexp(-_Complex_I * g * hs_eta(fields[(size_t)(t - 1) * N + x]));
        for (int y = 0; y < N; ++y) X[(size_t)x * N + y] *= ev;
      }
  }
  cudv_finish(N, X, u);
  free(X); free(Y);
}

/* G = (1 + B(tau,0) B(beta,tau))^-1 from the right chain R = B(tau,0) and the
 * left chain Lf = B(beta,tau)^H by scale separation (the complex form of the
 * stable G), with log|det(1 + B)| and its argument.  G_out [N][N] complex
 * (re, im interleaved). */
static int cudv_green(int N, const cudv_t* R, const cudv_t* Lf, double* G_out, double* logabs, double* arg) {
  const size_t NN = (size_t)N * N;
  double complex* Mid = (double complex*)calloc(NN, sizeof(double complex));
  double complex* X = (double complex*)calloc(NN, sizeof(double complex));
  double *dbR = dalloc(N), *dsR = dalloc(N), *dbL = dalloc(N), *dsL = dalloc(N);
  for (int i = 0; i < N; ++i) {
    dbR[i] = R->D[i] > 1.0 ? R->D[i] : 1.0;  dsR[i] = R->D[i] > 1.0 ? 1.0 : R->D[i];
    dbL[i] = Lf->D[i] > 1.0 ? Lf->D[i] : 1.0; dsL[i] = Lf->D[i] > 1.0 ? 1.0 : Lf->D[i];
  }
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) {
      double complex qq = 0.0, tt = 0.0;
      for (int k = 0; k < N; ++k) {
        qq += conj(R->Q[(size_t)k * N + i]) * Lf->Q[(size_t)k * N + j];   /* Q_R^H Q_L */
        tt += R->T[(size_t)i * N + k] * conj(Lf->T[(size_t)j * N + k]);   /* T_R T_L^H */
      }
      Mid[(size_t)i * N + j] = qq / (dbR[i] * dbL[j]) + dsR[i] * tt * dsL[j];
      X[(size_t)i * N + j] = conj(R->Q[(size_t)j * N + i]) / dbR[i];    /* Db_R^-1 Q_R^H */
    }
  /* Gauss-Jordan: X <- Mid^-1 X, with the determinant of Mid */
  double la = 0.0, ar = 0.0;
  int st = ORC_OK;
  for (int k = 0; k < N; ++k) {
    int p = k;
    for (int i = k + 1; i < N; ++i)
      if (cabs(Mid[(size_t)i * N + k]) > cabs(Mid[(size_t)p * N + k])) p = i;
    if (cabs(Mid[(size_t)p * N + k]) == 0.0) { st = ORC_ESING; break; }
    if (p != k) {
      for (int j = 0; j < N; ++j) {
        double complex t = Mid[(size_t)k * N + j]; Mid[(size_t)k * N + j] = Mid[(size_t)p * N + j]; Mid[(size_t)p * N + j] = t;
        t = X[(size_t)k * N + j]; X[(size_t)k * N + j] = X[(size_t)p * N + j]; X[(size_t)p * N + j] = t;
      }
      ar += 3.14159265358979323846;
    }
    const double complex d = Mid[(size_t)k * N + k];
    la += log(cabs(d));
    ar += carg(d);
    for (int j = 0; j < N; ++j) { Mid[(size_t)k * N + j] /= d; X[(size_t)k * N + j] /= d; }
    for (int i = 0; i < N; ++i) {
      if (i == k) continue;
      const double complex f = Mid[(size_t)i * N + k];
      if (f == 0.0) continue;
      for (int j = 0; j < N; ++j) { Mid[(size_t)i * N + j] -= f * Mid[(size_t)k * N + j]; X[(size_t)i * N + j] -= f * X[(size_t)k * N + j]; }
    }
  }
  if (!st) {
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < N; ++j) X[(size_t)i * N + j] /= dbL[i];
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < N; ++j) {
        double complex acc = 0.0;
        for (int k = 0; k < N; ++k) acc += Lf->Q[(size_t)i * N + k] * X[(size_t)k * N + j];
        G_out[2 * ((size_t)i * N + j)] = creal(acc);
        G_out[2 * ((size_t)i * N + j) + 1] = cimag(acc);
      }
    for (int i = 0; i < N; ++i) la += log(dbR[i]) + log(dbL[i]);
    if (R->detQ * Lf->detQ < 0) ar += 3.14159265358979323846;
    *logabs = la;
    *arg = remainder(ar, 2.0 * 3.14159265358979323846);
  }
  free(Mid); free(X); free(dbR); free(dsR); free(dbL); free(dsL);
  return st;
}

/* G(tau) of one color of the SU(2) decoupling through the complex UDV chains
 * (chunks of n_wrap slices; a partial chunk closes each chain), with
 * log|det(1 + B(beta,0))| and its argument.  G_out [N][N] complex (re, im). */
int orc_su2_green_udv(int N, const double* K, double dtau, double U, int L, int n_wrap, const int8_t* fields,
                      int tau, double* G_out, double* logabs, double* arg) {
  if (N < 1 || L < 1 || n_wrap < 1 || tau < 0 || tau > L || !(dtau > 0.0) || !(U >= 0.0)) return ORC_EINVAL;
  const size_t NN = (size_t)N * N;
  const double g = sqrt(0.5 * dtau * U);
  double* E = dalloc(NN);
  orc_expm_sym(N, K, -dtau, E);
  cudv_t R, Lf;
  cudv_alloc(N, &R);
  cudv_alloc(N, &Lf);
  for (int t = 0; t < tau; t += n_wrap) cudv_step(N, E, g, fields, t, (t + n_wrap < tau) ? t + n_wrap : tau, 0, &R);
  for (int t = L; t > tau; t -= n_wrap) cudv_step(N, E, g, fields, (t - n_wrap > tau) ? t - n_wrap : tau, t, 1, &Lf);
  const int st = cudv_green(N, &R, &Lf, G_out, logabs, arg);
  free(E);
  cudv_free(&R); cudv_free(&Lf);
  return st;
}

/* Time-displaced Green functions of the SU(2) decoupling on fixed fields (one
 * color; the definitions of the real case with complex B):
 *   G(tau,0) = B(tau,0) G(0) = (B(tau,0)^-1 + B(beta,tau))^-1,
 *   G(0,tau) = -(1 - G(0)) B(tau,0)^-1,
 * from the right chain R = B(tau,0) and the left chain Lf = B(beta,tau)^H with
 * the middle matrix of cudv_green:
 *   G(tau,0) = Q_L Db_L^-1 Mid^-1 Ds_R T_R,
 *   G(0,tau) = -T_L^H Ds_L Mid^-1 Db_R^-1 Q_R^H.
 * Gt0, G0t: [N][N] complex (re, im interleaved). */
static int cudv_displaced(int N, const cudv_t* R, const cudv_t* Lf, double* Gt0, double* G0t) {
  const size_t NN = (size_t)N * N;
  double complex* Mid = (double complex*)calloc(NN, sizeof(double complex));
  double complex* MI = (double complex*)calloc(NN, sizeof(double complex));
  double complex* X = (double complex*)calloc(NN, sizeof(double complex));
  double *dbR = dalloc(N), *dsR = dalloc(N), *dbL = dalloc(N), *dsL = dalloc(N);
  for (int i = 0; i < N; ++i) {
    dbR[i] = R->D[i] > 1.0 ? R->D[i] : 1.0;  dsR[i] = R->D[i] > 1.0 ? 1.0 : R->D[i];
    dbL[i] = Lf->D[i] > 1.0 ? Lf->D[i] : 1.0; dsL[i] = Lf->D[i] > 1.0 ? 1.0 : Lf->D[i];
  }
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) {
      double complex qq = 0.0, tt = 0.0;
      for (int k = 0; k < N; ++k) {
        qq += conj(R->Q[(size_t)k * N + i]) * Lf->Q[(size_t)k * N + j];
        tt += R->T[(size_t)i * N + k] * conj(Lf->T[(size_t)j * N + k]);
      }
      Mid[(size_t)i * N + j] = qq / (dbR[i] * dbL[j]) + dsR[i] * tt * dsL[j];
      MI[(size_t)i * N + j] = (i == j) ? 1.0 : 0.0;
    }
  /* Gauss-Jordan with partial pivoting: MI <- Mid^-1 */
  int st = ORC_OK;
  for (int k = 0; k < N && !st; ++k) {
    int p = k;
    for (int i = k + 1; i < N; ++i)
      if (cabs(Mid[(size_t)i * N + k]) > cabs(Mid[(size_t)p * N + k])) p = i;
    if (cabs(Mid[(size_t)p * N + k]) == 0.0) { st = ORC_ESING; break; }
    for (int j = 0; j < N; ++j) {
      double complex t = Mid[(size_t)k * N + j]; Mid[(size_t)k * N + j] = Mid[(size_t)p * N + j]; Mid[(size_t)p * N + j] = t;
      t = MI[(size_t)k * N + j]; MI[(size_t)k * N + j] = MI[(size_t)p * N + j]; MI[(size_t)p * N + j] = t;
    }
    const double complex d = Mid[(size_t)k * N + k];
    for (int j = 0; j < N; ++j) { Mid[(size_t)k * N + j] /= d; MI[(size_t)k * N + j] /= d; }
    for (int i = 0; i < N; ++i) {
      if (i == k) continue;
      const double complex f = Mid[(size_t)i * N + k];
      if (f == 0.0) continue;
      for (int j = 0; j < N; ++j) { Mid[(size_t)i * N + j] -= f * Mid[(size_t)k * N + j]; MI[(size_t)i * N + j] -= f * MI[(size_t)k * N + j]; }
    }
  }
  if (!st) {
    /* G(tau,0) = Q_L (Db_L^-1 MI Ds_R) T_R */
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < N; ++j) X[(size_t)i * N + j] = MI[(size_t)i * N + j] / dbL[i] * dsR[j];
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < N; ++j) {
        double complex acc = 0.0;
        for (int k = 0; k < N; ++k) {
          double complex qx = 0.0;
          for (int l = 0; l < N; ++l) qx += Lf->Q[(size_t)i * N + l] * X[(size_t)l * N + k];
          acc += qx * R->T[(size_t)k * N + j];
        }
        Gt0[2 * ((size_t)i * N + j)] = creal(acc);
        Gt0[2 * ((size_t)i * N + j) + 1] = cimag(acc);
      }
    /* G(0,tau) = -T_L^H (Ds_L MI Db_R^-1) Q_R^H */
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < N; ++j) X[(size_t)i * N + j] = dsL[i] * MI[(size_t)i * N + j] / dbR[j];
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < N; ++j) {
        double complex acc = 0.0;
        for (int k = 0; k < N; ++k) {
          double complex tx = 0.0;
          for (int l = 0; l < N; ++l) tx += conj(Lf->T[(size_t)l * N + i]) * X[(size_t)l * N + k];
          acc += tx * conj(R->Q[(size_t)j * N + k]);
        }
        G0t[2 * ((size_t)i * N + j)] = -creal(acc);
        G0t[2 * ((size_t)i * N + j) + 1] = -cimag(acc);
      }
  }
  free(Mid); free(MI); free(X); free(dbR); free(dsR); free(dbL); free(dsL);
  return st;
}

/* G(tau,0) and G(0,tau) of one color of the SU(2) decoupling through the
 * complex UDV chains (chunks of n_wrap slices, a partial chunk closing each
 * chain).  Gt0, G0t: [N][N] complex (re, im). */
int orc_su2_green_displaced(int N, const double* K, double dtau, double U, int L, int n_wrap, const int8_t* fields,
                            int tau, double* Gt0, double* G0t) {
  if (N < 1 || L < 1 || n_wrap < 1 || tau < 0 || tau > L || !(dtau > 0.0) || !(U >= 0.0)) return ORC_EINVAL;
  const double g = sqrt(0.5 * dtau * U);
  double* E = dalloc((size_t)N * N);
  orc_expm_sym(N, K, -dtau, E);
  cudv_t R, Lf;
  cudv_alloc(N, &R);
  cudv_alloc(N, &Lf);
  for (int t = 0; t < tau; t += n_wrap) cudv_step(N, E, g, fields, t, (t + n_wrap < tau) ? t + n_wrap : tau, 0, &R);
  for (int t = L; t > tau; t -= n_wrap) cudv_step(N, E, g, fields, (t - n_wrap > tau) ? t - n_wrap : tau, t, 1, &Lf);
  const int st = cudv_displaced(N, &R, &Lf, Gt0, G0t);
  free(E);
  cudv_free(&R); cudv_free(&Lf);
  return st;
}

/* ---- SVD stabilisation (the compile-time alternative of Sec. 5, -DSTAB1) -- */
/* The same UDV chain with the decomposition M = X D = U S V^T by one-sided     */
/* Jacobi rotations (Hestenes): column pairs of M are rotated until mutually    */
/* orthogonal, S_j = |m_j|, U = M S^-1, and V accumulates the rotations; then   */
/* Q = U, D = S, T = V^T T_old, det Q from an LU of U.  One-sided Jacobi keeps  */
/* the relative accuracy of the small singular values of a column-scaled        */
/* matrix, which is what the scale separation needs.                            */
static void udv_finish_svd(int N, double* X, udv_t* u) {
  const size_t NN = (size_t)N * N;
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) X[i * N + j] *= u->D[j];
  double* V = dalloc(NN);
  mat_identity(N, V);
  for (int sweep = 0; sweep < 60; ++sweep) {
    int rotated = 0;
    for (int p = 0; p < N - 1; ++p)
      for (int q = p + 1; q < N; ++q) {
        double a = 0.0, b = 0.0, c = 0.0;
        for (int i = 0; i < N; ++i) {
          a += X[i * N + p] * X[i * N + p];
          b += X[i * N + q] * X[i * N + q];
          c += X[i * N + p] * X[i * N + q];
        }
        if (c == 0.0 || fabs(c) <= 1e-15 * sqrt(a * b)) continue;
        rotated = 1;
        const double zeta = (b - a) / (2.0 * c);
        const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
        for (int i = 0; i < N; ++i) {
          const double xp = X[i * N + p], xq = X[i * N + q];
          X[i * N + p] = cs * xp - sn * xq;
          X[i * N + q] = sn * xp + cs * xq;
          const double vp = V[i * N + p], vq = V[i * N + q];
          V[i * N + p] = cs * vp - sn * vq;
          V[i * N + q] = sn * vp + cs * vq;
        }
      }
    if (!rotated) break;
  }
  double* S = dalloc(N);
  for (int j = 0; j < N; ++j) {
    double s2 = 0.0;
    for (int i = 0; i < N; ++i) s2 += X[i * N + j] * X[i * N + j];
    S[j] = sqrt(s2);
    for (int i = 0; i < N; ++i) X[i * N + j] = (S[j] > 0.0) ? X[i * N + j] / S[j] : (i == j ? 1.0 : 0.0);
  }
  /* T' = V^T T */
  double* Tn = dalloc(NN);
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) {
      double acc = 0.0;
      for (int k = 0; k < N; ++k) acc += V[k * N + i] * u->T[k * N + j];
      Tn[i * N + j] = acc;
    }
  double ld;
  int sg;
  orc_logdet(N, X, &ld, &sg);
  memcpy(u->Q, X, NN * sizeof(double));
  memcpy(u->T, Tn, NN * sizeof(double));
  memcpy(u->D, S, (size_t)N * sizeof(double));
  u->detQ = sg;
  free(V); free(S); free(Tn);
}

/* G(tau) like orc_green_udv, every chain step decomposed by SVD. */
int orc_green_udv_svd(const orc_model* m, const int8_t* fields, int s, int tau, double* G, double* logdet,
                      int* sign) {
  model_t M;
  int st = model_load(m, &M);
  if (st) return st;
  if (s < 0 || s >= M.nfl || tau < 0 || tau > M.L) { model_free(&M); return ORC_EINVAL; }
  const int N = M.N, nw = M.nw;
  udv_t R, Lf;
  udv_alloc(N, &R); udv_alloc(N, &Lf);
  udv_identity(N, &R); udv_identity(N, &Lf);
  double* X = dalloc((size_t)N * N);
  for (int t = 0; t < tau; t += nw) {
    memcpy(X, R.Q, sizeof(double) * N * N);
    for (int u = t + 1; u <= ((t + nw < tau) ? t + nw : tau); ++u) apply_B_left(&M, fields, s, u, X);
    udv_finish_svd(N, X, &R);
  }
  for (int t = M.L; t > tau; t -= nw) {
    memcpy(X, Lf.Q, sizeof(double) * N * N);
    for (int u = t; u >= ((t - nw > tau) ? t - nw : tau) + 1; --u) apply_BT_left(&M, fields, s, u, X);
    udv_finish_svd(N, X, &Lf);
  }
  st = green_from_udv(N, &R, &Lf, G, logdet, sign);
  free(X);
  udv_free(&R); udv_free(&Lf);
  model_free(&M);
  return st;
}

/* ------------------------------------------------------------------------ */
/* SU(2) Hubbard model coupled to a transverse Ising field on bonds (the     */
/* second example model of Sec. 6, Hubbard-Ising on the square lattice).     */
/* On fixed fields -- four-valued HS fields l[tau][x] of the charge          */
/* decoupling and Ising spins s[tau][b] = +-1 in the Z basis -- the fermion  */
/* propagator of one color is                                                */
/*   B_tau = exp(-dtau T) X_0 X_1 ... X_{nb-1} exp(V_tau),                    */
/*   X_b = exp(-dtau xi s_b O_b), O_b = |i><j| + |j><i| on bond b = (i, j),   */
/*   V_tau = diag(i g eta(l_tau,x)), g = sqrt(dtau U / 2),                    */
/* (the two-site type-1 operators of the bond terms: X_b acts on a 2 x 2     */
/* block as cosh(a) 1 + sinh(a) O, a = -dtau xi s_b).  Plain product, small  */
/* beta.  Outputs as orc_su2_plain; kin = 2 sum_xy T_xy (delta_xy - G_yx).    */
/* ------------------------------------------------------------------------ */
int orc_hubbard_ising_plain(int N, const double* T, int nb, const int32_t* bi, const int32_t* bj, double xi,
                            double dtau, double U, int L, const int8_t* hs, const int8_t* sz, double* G_out,
                            double* logabs, double* arg, double* phase, double* kin) {
  if (N < 1 || L < 1 || nb < 0 || !(dtau > 0.0) || !(U >= 0.0)) return ORC_EINVAL;
  for (int b = 0; b < nb; ++b)
    if (bi[b] < 0 || bi[b] >= N || bj[b] < 0 || bj[b] >= N || bi[b] == bj[b]) return ORC_EINVAL;
  const size_t NN = (size_t)N * N;
  double* E = dalloc(NN);
  orc_expm_sym(N, T, -dtau, E);
  double complex* B = (double complex*)calloc(NN, sizeof(double complex));
  double complex* Y = (double complex*)calloc(NN, sizeof(double complex));
  for (int x = 0; x < N; ++x) B[(size_t)x * N + x] = 1.0;
  const double g = sqrt(0.5 * dtau * U);
  double ph = 0.0;
  for (int tau = 1; tau <= L; ++tau) {
    /* B <- exp(V_tau) B */
    for (int x = 0; x < N; ++x) {
      const double th = g * hs_eta(hs[(size_t)(tau - 1) * N + x]);
      ph -= th;
      const double complex ev = cexp(_Complex_I * th);
      for (int y = 0; y < N; ++y) B[(size_t)x * N + y] *= ev;
    }
    /* B <- X_0 ... X_{nb-1} B: the last bond acts first */
    for (int b = nb - 1; b >= 0; --b) {
      const double a = -dtau * xi * (double)sz[(size_t)(tau - 1) * nb + b];
      const double ch = cosh(a), sh = sinh(a);
      const int i = bi[b], j = bj[b];
      for (int y = 0; y < N; ++y) {
        const double complex ri = B[(size_t)i * N + y], rj = B[(size_t)j * N + y];
        B[(size_t)i * N + y] = ch * ri + sh * rj;
        B[(size_t)j * N + y] = sh * ri + ch * rj;
      }
    }
    /* B <- E B */
    for (int x = 0; x < N; ++x)
      for (int y = 0; y < N; ++y) {
        double complex acc = 0.0;
        for (int k = 0; k < N; ++k) acc += E[(size_t)x * N + k] * B[(size_t)k * N + y];
        Y[(size_t)x * N + y] = acc;
      }
    memcpy(B, Y, NN * sizeof(double complex));
  }
  /* G = (1 + B)^-1 by Gauss-Jordan, with det(1 + B) */
  for (int x = 0; x < N; ++x) B[(size_t)x * N + x] += 1.0;
  double complex* G = (double complex*)calloc(NN, sizeof(double complex));
  for (int x = 0; x < N; ++x) G[(size_t)x * N + x] = 1.0;
  double la = 0.0, ar = 0.0;
  int st = ORC_OK;
  for (int k = 0; k < N; ++k) {
    int p = k;
    for (int i = k + 1; i < N; ++i)
      if (cabs(B[(size_t)i * N + k]) > cabs(B[(size_t)p * N + k])) p = i;
    if (cabs(B[(size_t)p * N + k]) == 0.0) { st = ORC_ESING; break; }
    if (p != k) {
      for (int j = 0; j < N; ++j) {
        double complex t = B[(size_t)k * N + j]; B[(size_t)k * N + j] = B[(size_t)p * N + j]; B[(size_t)p * N + j] = t;
        t = G[(size_t)k * N + j]; G[(size_t)k * N + j] = G[(size_t)p * N + j]; G[(size_t)p * N + j] = t;
      }
      ar += 3.14159265358979323846;
    }
    const double complex d = B[(size_t)k * N + k];
    la += log(cabs(d));
    ar += carg(d);
    for (int j = 0; j < N; ++j) { B[(size_t)k * N + j] /= d; G[(size_t)k * N + j] /= d; }
    for (int i = 0; i < N; ++i) {
      if (i == k) continue;
      const double complex f = B[(size_t)i * N + k];
      for (int j = 0; j < N; ++j) { B[(size_t)i * N + j] -= f * B[(size_t)k * N + j]; G[(size_t)i * N + j] -= f * G[(size_t)k * N + j]; }
    }
  }
  if (!st) {
    double complex kn = 0.0;
    for (int x = 0; x < N; ++x)
      for (int y = 0; y < N; ++y) kn += 2.0 * T[(size_t)x * N + y] * ((x == y ? 1.0 : 0.0) - G[(size_t)y * N + x]);
    for (size_t e = 0; e < NN; ++e) { G_out[2 * e] = creal(G[e]); G_out[2 * e + 1] = cimag(G[e]); }
    *logabs = la;
    *arg = remainder(ar, 2.0 * 3.14159265358979323846);
    *phase = ph;
    kin[0] = creal(kn); kin[1] = cimag(kn);
  }
  free(E); free(B); free(Y); free(G);
  return st;
}

/* Log weight of the Ising field on bonds in imaginary time (the S0 of the
 * Ising terms -h sum X_b - J sum Z_b Z_b'): the transverse field between
 * slices, <s'|exp(dtau h X)|s> = cosh(dtau h) (s' = s) or sinh(dtau h), for
 * each bond and each pair of neighbouring slices (periodic in tau), and
 * exp(dtau J sum_pairs s_b s_b') within each slice.  pairs: [n_pairs][2]. */
int orc_ising_bond_logweight(int nb, int L, const int8_t* sz, double dtau, double h, double J, int n_pairs,
                             const int32_t* pairs, double* logw) {
  if (nb < 1 || L < 1 || !(dtau > 0.0) || !(h > 0.0)) return ORC_EINVAL;
  double lw = 0.0;
  for (int tau = 0; tau < L; ++tau) {
    const int8_t* s = sz + (size_t)tau * nb;
    const int8_t* sn = sz + (size_t)((tau + 1) % L) * nb;
    for (int b = 0; b < nb; ++b) lw += (s[b] == sn[b]) ? log(cosh(dtau * h)) : log(sinh(dtau * h));
    for (int q = 0; q < n_pairs; ++q) lw += dtau * J * (double)(s[pairs[2 * q]] * s[pairs[2 * q + 1]]);
  }
  *logw = lw;
  return ORC_OK;
}

/* ---- Markov chain of the Hubbard-Ising bond model (rank-2 bond updates) --- */
/* The propagator of orc_hubbard_ising_plain as a cyclic list of elementary    */
/* factors in the order they act: per slice tau = 1..L, part 0 = exp(V_tau)     */
/* (all HS sites, diagonal), parts 1..nb = the bond factors X_{nb-1}, ..., X_0, */
/* part nb+1 = exp(-dtau T).  The Green function seen by a vertex is the one    */
/* just after its factor acted:                                                */
/*   G~ = (1 + F_p F_{p-1} ... F_0 F_{n-1} ... F_{p+1})^-1,                      */
/* so that changing F_p -> (1 + Delta) F_p multiplies det(1 + B) by            */
/* det(1 + Delta (1 - G~)), restricted to the rows Delta touches.              */
typedef struct {
  int N, nb, L;
  const int32_t *bi, *bj;
  const double* E;
  double g, a0; /* HS coupling sqrt(dtau U / 2); bond coupling -dtau xi */
  const int8_t *hs, *sz;
} hi_model_t;

/* A <- F A for the factor of slice tau (1-based), part p. */
static void hi_apply_factor(const hi_model_t* m, int tau, int part, double complex* A, double complex* T) {
  const int N = m->N;
  if (part == 0) {
    for (int x = 0; x < N; ++x) {
      const double complex ev = cexp(_Complex_I * m->g * hs_eta(m->hs[(size_t)(tau - 1) * N + x]));
      for (int y = 0; y < N; ++y) A[(size_t)x * N + y] *= ev;
    }
  } else if (part <= m->nb) {
    const int b = m->nb - part;
    const double a = m->a0 * (double)m->sz[(size_t)(tau - 1) * m->nb + b];
    const double ch = cosh(a), sh = sinh(a);
    const int i = m->bi[b], j = m->bj[b];
    for (int y = 0; y < N; ++y) {
      const double complex ri = A[(size_t)i * N + y], rj = A[(size_t)j * N + y];
      A[(size_t)i * N + y] = ch * ri + sh * rj;
      A[(size_t)j * N + y] = sh * ri + ch * rj;
    }
  } else {
    for (int x = 0; x < N; ++x)
      for (int y = 0; y < N; ++y) {
        double complex acc = 0.0;
        for (int k = 0; k < N; ++k) acc += m->E[(size_t)x * N + k] * A[(size_t)k * N + y];
        T[(size_t)x * N + y] = acc;
      }
    memcpy(A, T, (size_t)N * N * sizeof(double complex));
  }
}

/* G = (1 + A)^-1 by Gauss-Jordan with partial pivoting (A is destroyed). */
static int c_inverse_one_plus(int N, double complex* A, double complex* G) {
  for (int x = 0; x < N; ++x) A[(size_t)x * N + x] += 1.0;
  for (size_t e = 0; e < (size_t)N * N; ++e) G[e] = 0.0;
  for (int x = 0; x < N; ++x) G[(size_t)x * N + x] = 1.0;
  for (int k = 0; k < N; ++k) {
    int p = k;
    for (int i = k + 1; i < N; ++i)
      if (cabs(A[(size_t)i * N + k]) > cabs(A[(size_t)p * N + k])) p = i;
    if (cabs(A[(size_t)p * N + k]) == 0.0) return ORC_ESING;
    for (int j = 0; j < N; ++j) {
      double complex t = A[(size_t)k * N + j]; A[(size_t)k * N + j] = A[(size_t)p * N + j]; A[(size_t)p * N + j] = t;
      t = G[(size_t)k * N + j]; G[(size_t)k * N + j] = G[(size_t)p * N + j]; G[(size_t)p * N + j] = t;
    }
    const double complex d = A[(size_t)k * N + k];
    for (int j = 0; j < N; ++j) { A[(size_t)k * N + j] /= d; G[(size_t)k * N + j] /= d; }
    for (int i = 0; i < N; ++i) {
      if (i == k) continue;
      const double complex f = A[(size_t)i * N + k];
      for (int j = 0; j < N; ++j) { A[(size_t)i * N + j] -= f * A[(size_t)k * N + j]; G[(size_t)i * N + j] -= f * G[(size_t)k * N + j]; }
    }
  }
  return ORC_OK;
}

static int hi_green_at(const hi_model_t* m, int tau, int part, double complex* G) {
  const int N = m->N, P = m->nb + 2, nF = m->L * P;
  const size_t NN = (size_t)N * N;
  double complex* A = (double complex*)calloc(NN, sizeof(double complex));
  double complex* T = (double complex*)calloc(NN, sizeof(double complex));
  for (int x = 0; x < N; ++x) A[(size_t)x * N + x] = 1.0;
  const int f = (tau - 1) * P + part;
  for (int step = 1; step <= nF; ++step) {
    const int idx = (f + step) % nF;
    hi_apply_factor(m, idx / P + 1, idx % P, A, T);
  }
  const int st = c_inverse_one_plus(N, A, G);
  free(A); free(T);
  return st;
}

static int hi_model_init(hi_model_t* m, int N, const double* T, int nb, const int32_t* bi, const int32_t* bj,
                         double xi, double dtau, double U, int L, const int8_t* hs, const int8_t* sz) {
  if (N < 1 || L < 1 || nb < 0 || !(dtau > 0.0) || !(U >= 0.0)) return ORC_EINVAL;
  for (int b = 0; b < nb; ++b)
    if (bi[b] < 0 || bi[b] >= N || bj[b] < 0 || bj[b] >= N || bi[b] == bj[b]) return ORC_EINVAL;
  double* E = dalloc((size_t)N * N);
  orc_expm_sym(N, T, -dtau, E);
  m->N = N; m->nb = nb; m->L = L; m->bi = bi; m->bj = bj; m->E = E;
  m->g = sqrt(0.5 * dtau * U); m->a0 = -dtau * xi; m->hs = hs; m->sz = sz;
  return ORC_OK;
}

/* The Green function seen by the factor (tau, part) of the bond model, from
 * scratch (plain products).  G_out: [N][N] complex (re, im interleaved). */
int orc_hubbard_ising_green_at(int N, const double* T, int nb, const int32_t* bi, const int32_t* bj, double xi,
                               double dtau, double U, int L, const int8_t* hs, const int8_t* sz, int tau, int part,
                               double* G_out) {
  if (tau < 1 || tau > L || part < 0 || part > nb + 1) return ORC_EINVAL;
  hi_model_t m;
  int st = hi_model_init(&m, N, T, nb, bi, bj, xi, dtau, U, L, hs, sz);
  if (st) return st;
  double complex* G = (double complex*)malloc((size_t)N * N * sizeof(double complex));
  st = hi_green_at(&m, tau, part, G);
  if (!st)
    for (size_t e = 0; e < (size_t)N * N; ++e) { G_out[2 * e] = creal(G[e]); G_out[2 * e + 1] = cimag(G[e]); }
  free(G); free((void*)m.E);
  return st;
}

/* Rank-2 update of G~ when the factor seen by G~ changes by F -> (1 + Delta) F,
 * Delta nonzero only on the rows and columns {i, j} (the 2 x 2 block delta):
 * with (1 - G~)_PP the 2 x 2 block of 1 - G~ on {i, j} and (1 - G~)_P: its rows,
 *   ratio = det(1 + delta (1 - G~)_PP),
 *   G~' = G~ - G~_:P (1 + delta (1 - G~)_PP)^-1 delta (1 - G~)_P:
 * (Woodbury, with B (1 + B)^-1 = 1 - G~).  G: [N][N] complex in/out, delta:
 * 2 x 2 complex (re, im interleaved), ratio: re, im. */
int orc_bond_rank2_update(int N, double* G, int i, int j, const double* delta, double* ratio) {
  if (N < 2 || i < 0 || j < 0 || i >= N || j >= N || i == j) return ORC_EINVAL;
  const int P[2] = {i, j};
  double complex d[4], h[4], S[4], Si[4];
  for (int e = 0; e < 4; ++e) d[e] = delta[2 * e] + _Complex_I * delta[2 * e + 1];
#define GC(x, y) (G[2 * ((size_t)(x) * N + (y))] + _Complex_I * G[2 * ((size_t)(x) * N + (y)) + 1])
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) h[2 * a + b] = (a == b ? 1.0 : 0.0) - GC(P[a], P[b]);
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) S[2 * a + b] = (a == b ? 1.0 : 0.0) + d[2 * a] * h[b] + d[2 * a + 1] * h[2 + b];
  const double complex det = S[0] * S[3] - S[1] * S[2];
  ratio[0] = creal(det); ratio[1] = cimag(det);
  if (cabs(det) == 0.0) return ORC_ESING;
  Si[0] = S[3] / det; Si[1] = -S[1] / det; Si[2] = -S[2] / det; Si[3] = S[0] / det;
  /* W = S^-1 delta (2 x 2); rows of (1 - G~) on P: R[a][y] = delta_{P_a y} - G~_{P_a y} */
  double complex Wm[4];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) Wm[2 * a + b] = Si[2 * a] * d[b] + Si[2 * a + 1] * d[2 + b];
  double complex* R = (double complex*)malloc(2 * (size_t)N * sizeof(double complex));
  double complex* C = (double complex*)malloc(2 * (size_t)N * sizeof(double complex));
  for (int a = 0; a < 2; ++a)
    for (int y = 0; y < N; ++y) {
      R[(size_t)a * N + y] = (P[a] == y ? 1.0 : 0.0) - GC(P[a], y);
      C[(size_t)a * N + y] = GC(y, P[a]);   /* column P_a of G~, stored as a row */
    }
  for (int x = 0; x < N; ++x)
    for (int y = 0; y < N; ++y) {
      double complex acc = 0.0;
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) acc += C[(size_t)a * N + x] * Wm[2 * a + b] * R[(size_t)b * N + y];
      const size_t e = (size_t)x * N + y;
      G[2 * e] -= creal(acc);
      G[2 * e + 1] -= cimag(acc);
    }
#undef GC
  free(R); free(C);
  return ORC_OK;
}

/* One sweep of a Markov chain of the bond model: the four-valued HS fields and
 * the bond Ising spins are both updated, with W(C) = |Re e^{-S(C)}| (Sec. 2.2)
 * including the bond spins' own weight (the ratio S0 of Sec. 6 on a flip).
 * Order: up tau = 1..L, within a slice the factors in the order they act
 * (sites 0..N-1, then bonds nb-1..0); down tau = L..1 in the reverse order.
 * Random numbers as orc_su2_sweep, vertex index x for site x and N + b for
 * bond b (a bond proposal is the flip s -> -s and uses u2 only).  Ratios, G~
 * recomputed from scratch at each vertex:
 *   site:  gamma(l')/gamma(l) e^{-i g (eta'-eta)} (1 + Delta (1 - G~_xx))^2
 *   bond:  det(1 + delta (1 - G~)_PP)^2 * e^{logw(s') - logw(s)},
 *          delta = X_b(-2a) - 1 on the bond's 2 x 2 block, a = -dtau xi s_b.
 * After the sweep, with sign and P as orc_su2_sweep: obs[0..1] = reweighted
 * Kin (re, im), obs[2] = sign, obs[3..4] = reweighted (sum_b s_b)^2 / nb
 * averaged over slices (re, im). */
int orc_hubbard_ising_sweep(int N, const double* T, int nb, const int32_t* bi, const int32_t* bj, double xi, double h,
                            double J, int n_pairs, const int32_t* pairs, double dtau, double U, int L, int8_t* hs,
                            int8_t* sz, uint64_t seed, uint32_t chain, uint64_t sweep, double* phase, double* obs,
                            int* accepted) {
  if (nb < 1 || !(h > 0.0)) return ORC_EINVAL;
  hi_model_t m;
  int st = hi_model_init(&m, N, T, nb, bi, bj, xi, dtau, U, L, hs, sz);
  if (st) return st;
  const size_t NN = (size_t)N * N;
  double complex* Gt = (double complex*)malloc(NN * sizeof(double complex));
  double* Gd = dalloc(2 * NN);
  double la, ar, ph, kin[2];
  double complex P = phase[0] + _Complex_I * phase[1];
  if (phase[0] == 0.0 && phase[1] == 0.0) {
    st = orc_hubbard_ising_plain(N, T, nb, bi, bj, xi, dtau, U, L, hs, sz, Gd, &la, &ar, &ph, kin);
    P = cexp(_Complex_I * (ph + 2.0 * ar));
  }
  int acc = 0;
  const int nv = N + nb;
  for (int dir = 0; dir < 2 && !st; ++dir) {
    for (int step = 0; step < L && !st; ++step) {
      const int tau = dir ? L - step : step + 1;
      for (int q = 0; q < nv && !st; ++q) {
        const int v = dir ? nv - 1 - q : q;          /* position in the order the factors act */
        double u1, u2;
        double complex R;
        if (v < N) {
          const int x = v;
          proposal_uniforms(seed, chain, sweep, tau, dir, x, &u1, &u2);
          const int f = hs[(size_t)(tau - 1) * N + x];
          int others[3], n = 0;
          const int all[4] = {-2, -1, 1, 2};
          for (int a = 0; a < 4; ++a) if (all[a] != f) others[n++] = all[a];
          int idx = (int)floor(3.0 * u1);
          if (idx > 2) idx = 2;
          const int fn = others[idx];
          st = hi_green_at(&m, tau, 0, Gt);
          if (st) break;
          const double dth = m.g * (hs_eta(fn) - hs_eta(f));
          const double complex r1 = 1.0 + (cexp(_Complex_I * dth) - 1.0) * (1.0 - Gt[(size_t)x * N + x]);
          R = hs_gamma(fn) / hs_gamma(f) * cexp(-_Complex_I * dth) * r1 * r1;
          const double rr = fabs(creal(P * R)) / fabs(creal(P));
          if (u2 < (rr < 1.0 ? rr : 1.0)) {
            hs[(size_t)(tau - 1) * N + x] = (int8_t)fn;
            P = P * R / cabs(P * R);
            ++acc;
          }
        } else {
          const int b = nb - 1 - (v - N);            /* parts 1..nb act as bonds nb-1..0 */
          proposal_uniforms(seed, chain, sweep, tau, dir, N + b, &u1, &u2);
          st = hi_green_at(&m, tau, v - N + 1, Gt);
          if (st) break;
          int8_t* s = &sz[(size_t)(tau - 1) * nb + b];
          const double a = m.a0 * (double)(*s);
          const double delta[8] = {cosh(2.0 * a) - 1.0, 0.0, -sinh(2.0 * a), 0.0,
                                   -sinh(2.0 * a), 0.0, cosh(2.0 * a) - 1.0, 0.0};
          double* Gi = dalloc(2 * NN);
          for (size_t e = 0; e < NN; ++e) { Gi[2 * e] = creal(Gt[e]); Gi[2 * e + 1] = cimag(Gt[e]); }
          double r1[2];
          st = orc_bond_rank2_update(N, Gi, bi[b], bj[b], delta, r1);
          free(Gi);
          if (st == ORC_ESING) st = ORC_OK;            /* a zero ratio is a rejected proposal */
          if (st) break;
          double lw0, lw1;
          orc_ising_bond_logweight(nb, L, sz, dtau, h, J, n_pairs, pairs, &lw0);
          *s = (int8_t)(-*s);
          orc_ising_bond_logweight(nb, L, sz, dtau, h, J, n_pairs, pairs, &lw1);
          *s = (int8_t)(-*s);
          const double complex rf = r1[0] + _Complex_I * r1[1];
          R = rf * rf * exp(lw1 - lw0);
          const double rr = fabs(creal(P * R)) / fabs(creal(P));
          if (u2 < (rr < 1.0 ? rr : 1.0)) {
            *s = (int8_t)(-*s);
            P = P * R / cabs(P * R);
            ++acc;
          }
        }
      }
    }
  }
  if (!st) st = orc_hubbard_ising_plain(N, T, nb, bi, bj, xi, dtau, U, L, hs, sz, Gd, &la, &ar, &ph, kin);
  if (!st) {
    const double sgn = creal(P) >= 0.0 ? 1.0 : -1.0;
    const double complex rw = sgn * P / creal(P);
    const double complex wk = rw * (kin[0] + _Complex_I * kin[1]);
    double m2 = 0.0;
    for (int tau = 0; tau < L; ++tau) {
      double mt = 0.0;
      for (int b = 0; b < nb; ++b) mt += (double)sz[(size_t)tau * nb + b];
      m2 += mt * mt / (double)nb;
    }
    const double complex wm = rw * (m2 / (double)L);
    obs[0] = creal(wk); obs[1] = cimag(wk); obs[2] = sgn; obs[3] = creal(wm); obs[4] = cimag(wm);
    phase[0] = creal(P); phase[1] = cimag(P);
    *accepted = acc;
  }
  free(Gt); free(Gd); free((void*)m.E);
  return st;
}

/* ---- stable G of the bond model through the complex UDV chains ----------- */
/* Right chain X <- B_t X (factors in the order they act), left chain          */
/* X <- B_t^H X = F_0^H F_1^H ... F_{nb+1}^H X, where only the HS factor is not */
/* self-adjoint (its adjoint has e^{-i g eta}); chunks of n_wrap slices, the   */
/* complex QR steps and the scale-separated G of the SU(2) decoupling.         */
static void hi_udv_step(const hi_model_t* m, int t1, int t2, int left, cudv_t* u) {
  const int N = m->N;
  const size_t NN = (size_t)N * N;
  double complex* X = (double complex*)malloc(NN * sizeof(double complex));
  double complex* Y = (double complex*)malloc(NN * sizeof(double complex));
  memcpy(X, u->Q, NN * sizeof(double complex));
  for (int step = 0; step < t2 - t1; ++step) {
    const int t = left ? t2 - step : t1 + 1 + step;
    for (int q = 0; q <= m->nb + 1; ++q) {
      const int part = left ? m->nb + 1 - q : q;
      if (left && part == 0) {
        for (int x = 0; x < N; ++x) {
          const double complex ev = cexp(-_Complex_I * m->g * hs_eta(m->hs[(size_t)(t - 1) * N + x]));
          for (int y = 0; y < N; ++y) X[(size_t)x * N + y] *= ev;
        }
      } else {
        hi_apply_factor(m, t, part, X, Y);
      }
    }
  }
  cudv_finish(N, X, u);
  free(X); free(Y);
}

/* G(tau) = (1 + B(tau,0) B(beta,tau))^-1 of one color of the bond model at any
 * beta, with log|det(1 + B(beta,0))| and its argument.  G_out [N][N] complex. */
int orc_hubbard_ising_green_udv(int N, const double* T, int nb, const int32_t* bi, const int32_t* bj, double xi,
                                double dtau, double U, int L, int n_wrap, const int8_t* hs, const int8_t* sz, int tau,
                                double* G_out, double* logabs, double* arg) {
  if (n_wrap < 1 || tau < 0 || tau > L) return ORC_EINVAL;
  hi_model_t m;
  int st = hi_model_init(&m, N, T, nb, bi, bj, xi, dtau, U, L, hs, sz);
  if (st) return st;
  cudv_t R, Lf;
  cudv_alloc(N, &R);
  cudv_alloc(N, &Lf);
  for (int t = 0; t < tau; t += n_wrap) hi_udv_step(&m, t, (t + n_wrap < tau) ? t + n_wrap : tau, 0, &R);
  for (int t = L; t > tau; t -= n_wrap) hi_udv_step(&m, (t - n_wrap > tau) ? t - n_wrap : tau, t, 1, &Lf);
  st = cudv_green(N, &R, &Lf, G_out, logabs, arg);
  cudv_free(&R); cudv_free(&Lf);
  free((void*)m.E);
  return st;
}

/* Equal-time correlation functions of one configuration of the SU(2)
 * decoupling (the paper's default observables SpinZ, SpinXY, Den, Green,
 * collected per pair class).  Both colors see the same Green function G
 * (complex), so Wick's theorem gives, with X_xy = (delta_xy - G_yx) G_xy and
 * rho_x = 2 (1 - G_xx):
 *   <S^z_x S^z_y>        = X_xy / 2       (per configuration m_x = 0)
 *   <n_x n_y>            = rho_x rho_y + 2 X_xy
 *   <S^+_x S^-_y>        = X_xy
 *   sum_s <c^+_xs c_ys>  = 2 (delta_xy - G_yx)
 * G: [N][N] complex (re, im interleaved); out[(c * 4 + q) * 2 + {0, 1}] = re, im
 * of the class sums, classes as orc_correlations. */
int orc_su2_correlations(int N, const double* G, const int32_t* cls, int n_class, double* out) {
  if (N < 1 || n_class < 1) return ORC_EINVAL;
  for (int q = 0; q < 8 * n_class; ++q) out[q] = 0.0;
#define GZ(x, y) (G[2 * ((size_t)(x) * N + (y))] + _Complex_I * G[2 * ((size_t)(x) * N + (y)) + 1])
  for (int x = 0; x < N; ++x)
    for (int y = 0; y < N; ++y) {
      const int c = cls[x * N + y];
      if (c < 0) continue;
      if (c >= n_class) return ORC_EINVAL;
      const double dxy = (x == y) ? 1.0 : 0.0;
      const double complex hyx = dxy - GZ(y, x);
      const double complex X = hyx * GZ(x, y);
      const double complex rx = 2.0 * (1.0 - GZ(x, x)), ry = 2.0 * (1.0 - GZ(y, y));
      const double complex v[4] = {0.5 * X, rx * ry + 2.0 * X, X, 2.0 * hyx};
      for (int q = 0; q < 4; ++q) {
        out[(c * 4 + q) * 2] += creal(v[q]);
        out[(c * 4 + q) * 2 + 1] += cimag(v[q]);
      }
    }
#undef GZ
  return ORC_OK;
}
