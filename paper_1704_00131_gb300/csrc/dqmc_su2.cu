// GB300 kernels of the SU(2) charge decoupling of the Hubbard model, the
// paper's default Hubbard example (Sec. 6.1), in complex FP64.
//
// The discrete HS transform of Sec. 2.1 applied to exp(-dtau U/2 (n_i - 1)^2)
// has an imaginary coupling: on fixed four-valued fields l[tau][x] both colors
// see the same one-body propagator
//   B_tau = E exp(V_tau),  V_tau = diag(i g eta(l_tau,x)),  g = sqrt(dtau U / 2),
// and the weight is prod gamma(l)/4 * exp(-i g sum eta(l)) * det(1 + B(beta,0))^2.
// The Markov chain samples W = |Re e^{-S}| and carries the phase
// P = e^{-S} / |e^{-S}| (Sec. 2.2); observables are reweighted by
// sign * P / Re P (Sec. 5.1, ZS and ZP).
//
// Work decomposition: one CTA of 256 threads per chain; the chain's Green
// function, UDV storage and workspace live in its own arena in HBM.
// Per slice (Algorithm 1, wrapgrup): the V wrap G~ = e^V G e^-V, the
// sequential single-site updates with the complex ratio and a rank-1
// Sherman-Morrison update, the T wrap E G~ E^-1; every n_wrap slices the
// complex pivoted-QR UDV chain (Sec. 2.3) recomputes G, log|det|, the
// argument of det(1 + B) and with it the phase ("Precision Phase").
//
// Bond model (the Hubbard-Ising example of Sec. 6): Ising spins s_b on bonds
// couple to the hopping through two-site type-1 factors
// X_b = exp(-dtau xi s_b O_b), O_b = |i><j| + |j><i|, so that
// B_tau = E X_0 X_1 ... X_{nb-1} exp(V_tau).  The factors act in the order
// exp(V), X_{nb-1}, ..., X_0, E; each vertex sees the Green function just after
// its own factor acted.  A bond flip s -> -s changes its factor by
// (1 + Delta) with Delta = X(-2a) - 1 on the bond's 2 x 2 block: the ratio per
// color is det(1 + delta (1 - G~)_PP) and G~ takes a rank-2 (Woodbury) update;
// the spins' own weight (transverse field h between slices, coupling J between
// paired bonds; the S0 ratio of Sec. 6) multiplies the ratio.
#include "dqmc_device.cuh"
#include "dqmc_su2_internal.h"

namespace dqmc {
namespace {

// ---- complex arithmetic on double2 (re, im) -------------------------------
__device__ __forceinline__ double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 zsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 zconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 zscal(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
__device__ __forceinline__ double zabs2(double2 a) { return fma(a.x, a.x, a.y * a.y); }
__device__ __forceinline__ double zabs(double2 a) { return hypot(a.x, a.y); }
__device__ __forceinline__ double2 zdiv(double2 a, double2 b) {
  // a conj(b) / |b|^2 with b rescaled by its larger component (Smith's idea)
  const double s = fmax(fabs(b.x), fabs(b.y));
  const double2 bs = make_double2(b.x / s, b.y / s);
  const double d = zabs2(bs);
  const double2 n = zmul(a, zconj(bs));
  return make_double2(n.x / (d * s), n.y / (d * s));
}
__device__ __forceinline__ double2 zexpi(double th) {
  double s, c;
  sincos(th, &s, &c);
  return make_double2(c, s);
}
// acc + a b for complex and mixed real/complex operands
__device__ __forceinline__ double2 zmac(double2 acc, double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, acc.x)), fma(a.x, b.y, fma(a.y, b.x, acc.y)));
}
__device__ __forceinline__ double2 zmac(double2 acc, double a, double2 b) {
  return make_double2(fma(a, b.x, acc.x), fma(a, b.y, acc.y));
}
__device__ __forceinline__ double2 zmac(double2 acc, double2 a, double b) {
  return make_double2(fma(a.x, b, acc.x), fma(a.y, b, acc.y));
}
template <typename T>
__device__ __forceinline__ T zzero();
template <>
__device__ __forceinline__ double zzero<double>() { return 0.0; }
template <>
__device__ __forceinline__ double2 zzero<double2>() { return make_double2(0.0, 0.0); }
// operand transform: 0 as is, 1 transpose, 2 conjugate transpose
template <int OP>
__device__ __forceinline__ double zop(double x) { return x; }
template <int OP>
__device__ __forceinline__ double2 zop(double2 x) { return OP == 2 ? zconj(x) : x; }

__device__ __forceinline__ double2 block_zsum(double2 v, double* red) {
  const double re = block_sum(v.x, red);
  const double im = block_sum(v.y, red);
  return make_double2(re, im);
}

// ---- shared memory of a chain's CTA ----------------------------------------
constexpr int kZgTile = 32;  // C tile of the complex products
constexpr int kZgK = 16;     // K step
constexpr int kZgBytes = 2 * kZgK * (kZgTile + 1) * (int)sizeof(double2);

struct Sm {
  unsigned char* gemm;  // the two staging tiles of zgemm
  double2* ph;          // [N] exp(i g eta) of the current slice
  double2* delta;       // [N] e^{i dtheta} - 1 per proposal
  double2* gr;          // [N] gamma(l') / gamma(l) e^{-i dtheta} per proposal
  double2* d;           // [N] diagonal of G~
  double2* col;         // [N] column of G~ at the accepted site
  double2* row;         // [N] e_k - G~[k, :]
  double2* hv;          // [N] Householder vector; pivot column of Gauss-Jordan
  double2* qred;        // [8][32] partial sums of the reflector application
  double* u2;           // [N] acceptance uniforms
  double* red;          // [32]
  int* ired;            // [32]
  double2* P;           // [1] the phase of the chain
  int* first;           // [1] first accepted position of a scan
  int8_t* fsl;          // [MV] fields of the current slice (sites, then bonds)
  int8_t* fn;           // [N] proposed fields
};

__host__ __device__ inline size_t su2_smem_layout(int N, int MV) {
  return (size_t)kZgBytes + (size_t)8 * N * sizeof(double2) + 256 * sizeof(double2) + (size_t)N * sizeof(double) +
         32 * sizeof(double) + 32 * sizeof(int) + 16 /* alignment */ + sizeof(double2) + 16 +
         (size_t)((MV + 15) / 16 * 16) + (size_t)((N + 15) / 16 * 16);
}

__device__ inline Sm su2_carve(unsigned char* base, int N, int MV) {
  Sm s;
  unsigned char* q = base;
  s.gemm = q; q += kZgBytes;
  s.ph = reinterpret_cast<double2*>(q); q += (size_t)N * sizeof(double2);
  s.delta = reinterpret_cast<double2*>(q); q += (size_t)N * sizeof(double2);
  s.gr = reinterpret_cast<double2*>(q); q += (size_t)N * sizeof(double2);
  s.d = reinterpret_cast<double2*>(q); q += (size_t)N * sizeof(double2);
  s.col = reinterpret_cast<double2*>(q); q += (size_t)N * sizeof(double2);
  s.row = reinterpret_cast<double2*>(q); q += (size_t)N * sizeof(double2);
  s.hv = reinterpret_cast<double2*>(q); q += (size_t)N * sizeof(double2);
  q += (size_t)N * sizeof(double2);  // spare vector (keeps the layout 16-byte aligned)
  s.qred = reinterpret_cast<double2*>(q); q += 256 * sizeof(double2);
  s.u2 = reinterpret_cast<double*>(q); q += (size_t)N * sizeof(double);
  s.red = reinterpret_cast<double*>(q); q += 32 * sizeof(double);
  s.ired = reinterpret_cast<int*>(q); q += 32 * sizeof(int);
  q = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(q) + 15) & ~(uintptr_t)15);
  s.P = reinterpret_cast<double2*>(q); q += sizeof(double2);
  s.first = reinterpret_cast<int*>(q); q += 16;
  s.fsl = reinterpret_cast<int8_t*>(q); q += (size_t)((MV + 15) / 16 * 16);
  s.fn = reinterpret_cast<int8_t*>(q);
  return s;
}

// ---- dense complex products -------------------------------------------------
// C = op(A) op(B) (ACC: C += op(A) op(B)), M x Nc, inner dimension Kd; op 0 as
// is, 1 transpose, 2 conjugate transpose; A and B real (double) or complex
// (double2).  Tiles of 32 x 32 outputs, 2 x 2 per thread, K in steps of 16
// staged in shared memory.  C must not alias A or B.
template <int OPA, int OPB, bool ACC, typename TA, typename TB>
__device__ void zgemm(int M, int Nc, int Kd, const TA* A, int lda, const TB* B, int ldb, double2* C, int ldc,
                      unsigned char* smem) {
  TA* As = reinterpret_cast<TA*>(smem);                                     // [kZgK][33] (k, m)
  TB* Bs = reinterpret_cast<TB*>(smem + kZgK * (kZgTile + 1) * sizeof(double2));  // [kZgK][33] (k, n)
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int mt = (M + kZgTile - 1) / kZgTile, nt = (Nc + kZgTile - 1) / kZgTile;
  for (int t = 0; t < mt * nt; ++t) {
    const int m0 = (t / nt) * kZgTile, n0 = (t % nt) * kZgTile;
    double2 acc[2][2];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int c = 0; c < 2; ++c) acc[r][c] = make_double2(0.0, 0.0);
    for (int k0 = 0; k0 < Kd; k0 += kZgK) {
      for (int e = tid; e < kZgTile * kZgK; e += kThreads) {
        int mm, kk;
        if (OPA == 0) { mm = e >> 4; kk = e & 15; } else { kk = e >> 5; mm = e & 31; }
        const int gm = m0 + mm, gk = k0 + kk;
        TA v = zzero<TA>();
        if (gm < M && gk < Kd) v = (OPA == 0) ? A[(size_t)gm * lda + gk] : zop<OPA>(A[(size_t)gk * lda + gm]);
        As[kk * (kZgTile + 1) + mm] = v;
      }
      for (int e = tid; e < kZgTile * kZgK; e += kThreads) {
        int nn, kk;
        if (OPB == 0) { kk = e >> 5; nn = e & 31; } else { nn = e >> 4; kk = e & 15; }
        const int gn = n0 + nn, gk = k0 + kk;
        TB v = zzero<TB>();
        if (gn < Nc && gk < Kd) v = (OPB == 0) ? B[(size_t)gk * ldb + gn] : zop<OPB>(B[(size_t)gn * ldb + gk]);
        Bs[kk * (kZgTile + 1) + nn] = v;
      }
      __syncthreads();
#pragma unroll 4
      for (int kk = 0; kk < kZgK; ++kk) {
        const TA a0 = As[kk * (kZgTile + 1) + 2 * ty], a1 = As[kk * (kZgTile + 1) + 2 * ty + 1];
        const TB b0 = Bs[kk * (kZgTile + 1) + 2 * tx], b1 = Bs[kk * (kZgTile + 1) + 2 * tx + 1];
        acc[0][0] = zmac(acc[0][0], a0, b0);
        acc[0][1] = zmac(acc[0][1], a0, b1);
        acc[1][0] = zmac(acc[1][0], a1, b0);
        acc[1][1] = zmac(acc[1][1], a1, b1);
      }
      __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int gm = m0 + 2 * ty + r, gn = n0 + 2 * tx + c;
        if (gm < M && gn < Nc) {
          double2* cp = C + (size_t)gm * ldc + gn;
          *cp = ACC ? zadd(*cp, acc[r][c]) : acc[r][c];
        }
      }
  }
  __syncthreads();
}

__device__ inline void zcopy(int N, int ld, const double2* src, double2* dst) {
  for (int e = threadIdx.x; e < N * N; e += kThreads) {
    const int x = e / N, y = e - x * N;
    dst[(size_t)x * ld + y] = src[(size_t)x * ld + y];
  }
  __syncthreads();
}

// ---- per-chain workspace --------------------------------------------------
__device__ inline double2* zmat(const Su2Dev& C, int m) { return C.work + (size_t)m * C.N * C.ld; }
__device__ inline double2* zvec(const Su2Dev& C, int v) {
  return C.work + (size_t)kSu2Mats * C.N * C.ld + (size_t)v * C.ld;
}
__device__ inline double* dvec(const Su2Dev& C, int v) { return C.dwork + (size_t)v * C.ld; }

struct ZUdv {
  const double2* Q;
  const double* D;
  const double2* T;
  int detq;
};
__device__ inline ZUdv z_ident(const Su2Dev& C) { return ZUdv{C.ident, C.ones, C.ident, 1}; }
__device__ inline ZUdv z_slot(const Su2Dev& C, int j) {
  const double2* b = C.slots + (size_t)j * su2_slot_elems(C.N, C.ld);
  return ZUdv{b, C.slotD + (size_t)j * C.ld, b + (size_t)C.N * C.ld, C.slot_detq[j]};
}
// the decomposition a chain step leaves in the workspace: Q in W2, T in W3, D in dvec 0
__device__ inline ZUdv z_work(const Su2Dev& C, int detq) { return ZUdv{zmat(C, 2), dvec(C, 0), zmat(C, 3), detq}; }
__device__ void z_store_slot(const Su2Dev& C, int j, int detq) {
  const int N = C.N, ld = C.ld;
  double2* b = C.slots + (size_t)j * su2_slot_elems(N, ld);
  zcopy(N, ld, zmat(C, 2), b);
  zcopy(N, ld, zmat(C, 3), b + (size_t)N * ld);
  for (int x = threadIdx.x; x < N; x += kThreads) C.slotD[(size_t)j * ld + x] = dvec(C, 0)[x];
  if (threadIdx.x == 0) C.slot_detq[j] = detq;
  __syncthreads();
}

// exp(s i g eta(l)) of slice tau for every site, into ph (s = +1 or -1)
__device__ inline void slice_phases(const Su2Dev& C, const int8_t* f, double s, double2* ph) {
  for (int x = threadIdx.x; x < C.N; x += kThreads) ph[x] = zexpi(s * C.g * hs_eta(f[x]));
  __syncthreads();
}

// A <- X_b(a) A: rows i, j of A mixed by [[cosh a, sinh a], [sinh a, cosh a]]
__device__ void bond_rows(int N, int ld, double2* A, int i, int j, double a) {
  const double ch = cosh(a), sh = sinh(a);
  for (int y = threadIdx.x; y < N; y += kThreads) {
    const double2 ri = A[(size_t)i * ld + y], rj = A[(size_t)j * ld + y];
    A[(size_t)i * ld + y] = zadd(zscal(ch, ri), zscal(sh, rj));
    A[(size_t)j * ld + y] = zadd(zscal(sh, ri), zscal(ch, rj));
  }
  __syncthreads();
}
// A <- A X_b(a): columns i, j of A mixed the same way (X_b is symmetric)
__device__ void bond_cols(int N, int ld, double2* A, int i, int j, double a) {
  const double ch = cosh(a), sh = sinh(a);
  for (int x = threadIdx.x; x < N; x += kThreads) {
    const double2 ci = A[(size_t)x * ld + i], cj = A[(size_t)x * ld + j];
    A[(size_t)x * ld + i] = zadd(zscal(ch, ci), zscal(sh, cj));
    A[(size_t)x * ld + j] = zadd(zscal(sh, ci), zscal(ch, cj));
  }
  __syncthreads();
}

// ---- complex Householder QR with column pivoting ---------------------------
// X[k:, j] -= b v (v^H X[k:, j]) for j0 <= j < N, v = hv[k:], b real.  8 row
// groups x 32 columns; the row groups' partial products are summed in shared
// memory in a fixed order.
__device__ void zhouse_apply(int N, int ld, double2* X, int k, int j0, double b, const double2* hv,
                             double2* qred) {
  const int tid = threadIdx.x, lane = tid & 31, rg = tid >> 5;
  for (int c0 = j0; c0 < N; c0 += 32) {
    const int j = c0 + lane;
    double2 w = make_double2(0.0, 0.0);
    if (j < N)
      for (int i = k + rg; i < N; i += 8) w = zmac(w, zconj(hv[i]), X[(size_t)i * ld + j]);
    qred[rg * 32 + lane] = w;
    __syncthreads();
    double2 s = make_double2(0.0, 0.0);
#pragma unroll
    for (int r = 0; r < 8; ++r) s = zadd(s, qred[r * 32 + lane]);
    s = zscal(b, s);
    if (j < N)
      for (int i = k + rg; i < N; i += 8) {
        double2* xp = X + (size_t)i * ld + j;
        *xp = zsub(*xp, zmul(s, hv[i]));
      }
    __syncthreads();
  }
}

// Pivoted QR of X (in place): the upper triangle becomes R, the strict lower
// part keeps the reflector vectors below their first entries (vk0[k]);
// H_k = 1 - beta_k v v^H maps column k of the remaining block to alpha e_k with
// alpha = -(x_0/|x_0|) |x| (Hermitian, unitary, det -1).  The pivot is the
// column of largest remaining norm (ties: lowest index), the norms downdated
// as in LAPACK's xGEQPF and recomputed when cancellation would spoil them.
// perm[k] = the original column now at position k.  Returns det Q.
__device__ int zqr_pivoted(int N, int ld, double2* X, double* beta, double2* vk0, double* cn, double* cn0, int* perm,
                           Sm& S) {
  const int tid = threadIdx.x;
  for (int j = tid; j < N; j += kThreads) {
    double acc = 0.0;
    for (int i = 0; i < N; ++i) acc += zabs2(X[(size_t)i * ld + j]);
    cn[j] = sqrt(acc);
    cn0[j] = cn[j];
    perm[j] = j;
  }
  __syncthreads();
  const double tol3z = sqrt(2.220446049250313e-16);
  int detq = 1;
  for (int k = 0; k < N; ++k) {
    double bv = -1.0;
    int bi = N;
    for (int j = k + tid; j < N; j += kThreads)
      if (cn[j] > bv) { bv = cn[j]; bi = j; }
    int p = block_argmax(bv, bi, S.red, S.ired);
    if (p >= N) p = k;
    if (p != k) {
      for (int i = tid; i < N; i += kThreads) {
        const double2 t = X[(size_t)i * ld + k];
        X[(size_t)i * ld + k] = X[(size_t)i * ld + p];
        X[(size_t)i * ld + p] = t;
      }
      if (tid == 0) {
        const int tp = perm[k]; perm[k] = perm[p]; perm[p] = tp;
        double t = cn[k]; cn[k] = cn[p]; cn[p] = t;
        t = cn0[k]; cn0[k] = cn0[p]; cn0[p] = t;
      }
      __syncthreads();
    }
    double part = 0.0;
    for (int i = k + tid; i < N; i += kThreads) {
      const double2 x = X[(size_t)i * ld + k];
      part += zabs2(x);
      S.hv[i] = x;
    }
    const double xn2 = block_sum(part, S.red);
    const double xnorm = sqrt(xn2);
    const double2 x0 = S.hv[k];
    double bk = 0.0;
    double2 alpha = make_double2(0.0, 0.0);
    if (xnorm > 0.0) {
      const double a0 = zabs(x0);
      alpha = (a0 > 0.0) ? zscal(-xnorm / a0, x0) : make_double2(-xnorm, 0.0);
      const double2 v0 = zsub(x0, alpha);
      const double vhv = xn2 - zabs2(x0) + zabs2(v0);
      bk = (vhv > 0.0) ? 2.0 / vhv : 0.0;
      __syncthreads();
      if (tid == 0) S.hv[k] = v0;
      __syncthreads();
    }
    if (tid == 0) {
      beta[k] = bk;
      vk0[k] = S.hv[k];
    }
    if (bk != 0.0) {
      detq = -detq;
      zhouse_apply(N, ld, X, k, k + 1, bk, S.hv, S.qred);
    }
    __syncthreads();
    if (tid == 0) X[(size_t)k * ld + k] = (xnorm > 0.0) ? alpha : x0;
    for (int j = k + 1 + tid; j < N; j += kThreads) {
      if (cn[j] != 0.0) {
        double t = zabs(X[(size_t)k * ld + j]) / cn[j];
        t = fmax(0.0, (1.0 + t) * (1.0 - t));
        const double r = cn[j] / cn0[j];
        if (t * r * r <= tol3z) {
          double acc = 0.0;
          for (int i = k + 1; i < N; ++i) acc += zabs2(X[(size_t)i * ld + j]);
          cn[j] = sqrt(acc);
          cn0[j] = cn[j];
        } else {
          cn[j] *= sqrt(t);
        }
      }
    }
    __syncthreads();
  }
  return detq;
}

// Q = H_0 H_1 ... H_{N-1}, applied to the identity from the last reflector.
__device__ void zform_q(int N, int ld, const double2* X, const double* beta, const double2* vk0, double2* Q, Sm& S) {
  for (int e = threadIdx.x; e < N * N; e += kThreads) {
    const int x = e / N, y = e - x * N;
    Q[(size_t)x * ld + y] = make_double2(x == y ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  for (int k = N - 1; k >= 0; --k) {
    const double bk = beta[k];
    if (bk == 0.0) continue;
    for (int i = k + threadIdx.x; i < N; i += kThreads) S.hv[i] = (i == k) ? vk0[k] : X[(size_t)i * ld + k];
    __syncthreads();
    zhouse_apply(N, ld, Q, k, k, bk, S.hv, S.qred);
  }
}

// ---- the UDV chain (Sec. 2.3) -----------------------------------------------
// Extend a decomposition by the slices t1+1..t2.  Right chain (B(tau,0)):
// X <- B_t X = E e^{V_t} X for t = t1+1..t2.  Left chain (B(beta,tau)^H):
// X <- B_t^H X = e^{-V_t} E X for t = t2..t1+1.  Starting from X = src.Q, then
// M = X diag(src.D) = Q R P^T; the new decomposition is Q (W2), D = |diag R|
// (dvec 0), T = D^-1 R P^T src.T (W3).  Returns det Q.
__device__ int z_chain_step(const Su2Dev& C, int t1, int t2, bool left, ZUdv src, Sm& S) {
  const int N = C.N, ld = C.ld;
  double2* X = zmat(C, 0);
  double2* Y = zmat(C, 1);
  zcopy(N, ld, src.Q, X);
  for (int q = 0; q < t2 - t1; ++q) {
    const int t = left ? t2 - q : t1 + 1 + q;
    const int8_t* f = C.fields + (size_t)(t - 1) * C.MV;
    if (!left) {
      slice_phases(C, f, +1.0, S.ph);
      for (int e = threadIdx.x; e < N * N; e += kThreads) {
        const int x = e / N, y = e - x * N;
        X[(size_t)x * ld + y] = zmul(S.ph[x], X[(size_t)x * ld + y]);
      }
      __syncthreads();
      for (int b = C.nb - 1; b >= 0; --b) bond_rows(N, ld, X, C.bi[b], C.bj[b], C.a0 * f[N + b]);
      zgemm<0, 0, false>(N, N, N, C.E, ld, X, ld, Y, ld, S.gemm);
    } else {
      zgemm<0, 0, false>(N, N, N, C.E, ld, X, ld, Y, ld, S.gemm);
      for (int b = 0; b < C.nb; ++b) bond_rows(N, ld, Y, C.bi[b], C.bj[b], C.a0 * f[N + b]);
      slice_phases(C, f, -1.0, S.ph);
      for (int e = threadIdx.x; e < N * N; e += kThreads) {
        const int x = e / N, y = e - x * N;
        Y[(size_t)x * ld + y] = zmul(S.ph[x], Y[(size_t)x * ld + y]);
      }
      __syncthreads();
    }
    double2* t_ = X; X = Y; Y = t_;
  }
  // M = X diag(D)
  for (int e = threadIdx.x; e < N * N; e += kThreads) {
    const int x = e / N, y = e - x * N;
    X[(size_t)x * ld + y] = zscal(src.D[y], X[(size_t)x * ld + y]);
  }
  __syncthreads();
  double* Dn = dvec(C, 0);
  double* beta = dvec(C, 1);
  double2* vk0 = zvec(C, 0);
  int* perm = C.iwork;
  const int detq = zqr_pivoted(N, ld, X, beta, vk0, dvec(C, 2), dvec(C, 3), perm, S);
  zform_q(N, ld, X, beta, vk0, zmat(C, 2), S);
  for (int k = threadIdx.x; k < N; k += kThreads) Dn[k] = zabs(X[(size_t)k * ld + k]);
  __syncthreads();
  // Y = D^-1 R (upper triangle), Rt = P^T src.T (row k = row perm[k] of src.T)
  double2* Rt = zmat(C, 7);
  for (int e = threadIdx.x; e < N * N; e += kThreads) {
    const int x = e / N, y = e - x * N;
    const double dinv = Dn[x] > 0.0 ? 1.0 / Dn[x] : 0.0;
    Y[(size_t)x * ld + y] = (y >= x) ? zscal(dinv, X[(size_t)x * ld + y]) : make_double2(0.0, 0.0);
    Rt[(size_t)x * ld + y] = src.T[(size_t)perm[x] * ld + y];
  }
  __syncthreads();
  zgemm<0, 0, false>(N, N, N, (const double2*)Y, ld, (const double2*)Rt, ld, zmat(C, 3), ld, S.gemm);
  return detq;
}

// G = (1 + B(tau,0) B(beta,tau))^-1 from the right chain R = B(tau,0) and the
// left chain Lf = B(beta,tau)^H by scale separation (D = Db Ds with
// Db = max(D, 1), Ds = min(D, 1)):
//   1 + B(tau,0) B(beta,tau) = Q_R Db_R Mid Db_L Q_L^H,
//   Mid = Db_R^-1 Q_R^H Q_L Db_L^-1 + Ds_R T_R T_L^H Ds_L,
//   G = Q_L Db_L^-1 Mid^-1 Db_R^-1 Q_R^H,
//   det(1 + B) = det Q_R det Q_L prod Db_R prod Db_L det Mid (det Q = +-1).
// Mid^-1 by Gauss-Jordan with partial pivoting.  Returns 1 on a singular Mid.
__device__ int z_green(const Su2Dev& C, ZUdv R, ZUdv Lf, double2* Gout, double& logabs, double& arg, Sm& S) {
  const int N = C.N, ld = C.ld, tid = threadIdx.x;
  double *dbR = dvec(C, 4), *dsR = dvec(C, 5), *dbL = dvec(C, 6), *dsL = dvec(C, 7);
  double lsum = 0.0;
  for (int i = tid; i < N; i += kThreads) {
    dbR[i] = fmax(R.D[i], 1.0);
    dsR[i] = fmin(R.D[i], 1.0);
    dbL[i] = fmax(Lf.D[i], 1.0);
    dsL[i] = fmin(Lf.D[i], 1.0);
    lsum += log(dbR[i]) + log(dbL[i]);
  }
  lsum = block_sum(lsum, S.red);
  double2* Mid = zmat(C, 4);
  double2* X = zmat(C, 5);
  zgemm<2, 0, false>(N, N, N, R.Q, ld, Lf.Q, ld, Mid, ld, S.gemm);  // Q_R^H Q_L
  zgemm<0, 2, false>(N, N, N, R.T, ld, Lf.T, ld, X, ld, S.gemm);    // T_R T_L^H
  for (int e = tid; e < N * N; e += kThreads) {
    const int i = e / N, j = e - i * N;
    const double2 qq = Mid[(size_t)i * ld + j], tt = X[(size_t)i * ld + j];
    Mid[(size_t)i * ld + j] = zadd(zscal(1.0 / (dbR[i] * dbL[j]), qq), zscal(dsR[i] * dsL[j], tt));
  }
  __syncthreads();
  for (int e = tid; e < N * N; e += kThreads) {
    const int i = e / N, j = e - i * N;
    X[(size_t)i * ld + j] = zscal(1.0 / dbR[i], zconj(R.Q[(size_t)j * ld + i]));  // Db_R^-1 Q_R^H
  }
  __syncthreads();
  double la = 0.0, ar = 0.0;
  for (int k = 0; k < N; ++k) {
    double bv = -1.0;
    int bi = N;
    for (int i = k + tid; i < N; i += kThreads) {
      const double a = zabs(Mid[(size_t)i * ld + k]);
      if (a > bv) { bv = a; bi = i; }
    }
    const int p = block_argmax(bv, bi, S.red, S.ired);
    if (p >= N || zabs(Mid[(size_t)p * ld + k]) == 0.0) return 1;
    if (p != k) {
      for (int j = tid; j < N; j += kThreads) {
        double2 t = Mid[(size_t)k * ld + j]; Mid[(size_t)k * ld + j] = Mid[(size_t)p * ld + j]; Mid[(size_t)p * ld + j] = t;
        t = X[(size_t)k * ld + j]; X[(size_t)k * ld + j] = X[(size_t)p * ld + j]; X[(size_t)p * ld + j] = t;
      }
      ar += 3.14159265358979323846;
      __syncthreads();
    }
    const double2 d = Mid[(size_t)k * ld + k];
    la += log(zabs(d));
    ar += atan2(d.y, d.x);
    const double2 dinv = zdiv(make_double2(1.0, 0.0), d);
    __syncthreads();
    for (int j = tid; j < N; j += kThreads) {
      Mid[(size_t)k * ld + j] = zmul(Mid[(size_t)k * ld + j], dinv);
      X[(size_t)k * ld + j] = zmul(X[(size_t)k * ld + j], dinv);
    }
    for (int i = tid; i < N; i += kThreads) S.hv[i] = (i == k) ? make_double2(0.0, 0.0) : Mid[(size_t)i * ld + k];
    __syncthreads();
    for (int e = tid; e < N * N; e += kThreads) {
      const int i = e / N, j = e - i * N;
      if (i == k) continue;
      const double2 f = S.hv[i];
      Mid[(size_t)i * ld + j] = zsub(Mid[(size_t)i * ld + j], zmul(f, Mid[(size_t)k * ld + j]));
      X[(size_t)i * ld + j] = zsub(X[(size_t)i * ld + j], zmul(f, X[(size_t)k * ld + j]));
    }
    __syncthreads();
  }
  for (int e = tid; e < N * N; e += kThreads) {
    const int i = e / N, j = e - i * N;
    X[(size_t)i * ld + j] = zscal(1.0 / dbL[i], X[(size_t)i * ld + j]);
  }
  __syncthreads();
  zgemm<0, 0, false>(N, N, N, Lf.Q, ld, (const double2*)X, ld, Gout, ld, S.gemm);
  if (R.detq * Lf.detq < 0) ar += 3.14159265358979323846;
  logabs = la + lsum;
  arg = remainder(ar, 2.0 * 3.14159265358979323846);
  return 0;
}

// Time-displaced Green functions from the right chain R = B(tau,0) and the
// left chain Lf = B(beta,tau)^H, with the middle matrix of z_green:
//   G(tau,0) = (B(tau,0)^-1 + B(beta,tau))^-1 = Q_L Db_L^-1 Mid^-1 Ds_R T_R,
//   G(0,tau) = -(1 - G(0)) B(tau,0)^-1 = -T_L^H Ds_L Mid^-1 Db_R^-1 Q_R^H.
// Mid^-1 by Gauss-Jordan with partial pivoting.  Returns 1 on a singular Mid.
__device__ int z_displaced(const Su2Dev& C, ZUdv R, ZUdv Lf, double2* Gt0, double2* G0t, Sm& S) {
  const int N = C.N, ld = C.ld, tid = threadIdx.x;
  double *dbR = dvec(C, 4), *dsR = dvec(C, 5), *dbL = dvec(C, 6), *dsL = dvec(C, 7);
  for (int i = tid; i < N; i += kThreads) {
    dbR[i] = fmax(R.D[i], 1.0);
    dsR[i] = fmin(R.D[i], 1.0);
    dbL[i] = fmax(Lf.D[i], 1.0);
    dsL[i] = fmin(Lf.D[i], 1.0);
  }
  __syncthreads();
  double2* Mid = zmat(C, 4);
  double2* MI = zmat(C, 5);
  double2* X = zmat(C, 7);
  zgemm<2, 0, false>(N, N, N, R.Q, ld, Lf.Q, ld, Mid, ld, S.gemm);  // Q_R^H Q_L
  zgemm<0, 2, false>(N, N, N, R.T, ld, Lf.T, ld, X, ld, S.gemm);    // T_R T_L^H
  for (int e = tid; e < N * N; e += kThreads) {
    const int i = e / N, j = e - i * N;
    Mid[(size_t)i * ld + j] = zadd(zscal(1.0 / (dbR[i] * dbL[j]), Mid[(size_t)i * ld + j]),
                                   zscal(dsR[i] * dsL[j], X[(size_t)i * ld + j]));
    MI[(size_t)i * ld + j] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  for (int k = 0; k < N; ++k) {
    double bv = -1.0;
    int bi = N;
    for (int i = k + tid; i < N; i += kThreads) {
      const double a = zabs(Mid[(size_t)i * ld + k]);
      if (a > bv) { bv = a; bi = i; }
    }
    const int p = block_argmax(bv, bi, S.red, S.ired);
    if (p >= N || zabs(Mid[(size_t)p * ld + k]) == 0.0) return 1;
    if (p != k) {
      for (int j = tid; j < N; j += kThreads) {
        double2 t = Mid[(size_t)k * ld + j]; Mid[(size_t)k * ld + j] = Mid[(size_t)p * ld + j]; Mid[(size_t)p * ld + j] = t;
        t = MI[(size_t)k * ld + j]; MI[(size_t)k * ld + j] = MI[(size_t)p * ld + j]; MI[(size_t)p * ld + j] = t;
      }
      __syncthreads();
    }
    const double2 dinv = zdiv(make_double2(1.0, 0.0), Mid[(size_t)k * ld + k]);
    __syncthreads();
    for (int j = tid; j < N; j += kThreads) {
      Mid[(size_t)k * ld + j] = zmul(Mid[(size_t)k * ld + j], dinv);
      MI[(size_t)k * ld + j] = zmul(MI[(size_t)k * ld + j], dinv);
    }
    for (int i = tid; i < N; i += kThreads) S.hv[i] = (i == k) ? make_double2(0.0, 0.0) : Mid[(size_t)i * ld + k];
    __syncthreads();
    for (int e = tid; e < N * N; e += kThreads) {
      const int i = e / N, j = e - i * N;
      if (i == k) continue;
      const double2 f = S.hv[i];
      Mid[(size_t)i * ld + j] = zsub(Mid[(size_t)i * ld + j], zmul(f, Mid[(size_t)k * ld + j]));
      MI[(size_t)i * ld + j] = zsub(MI[(size_t)i * ld + j], zmul(f, MI[(size_t)k * ld + j]));
    }
    __syncthreads();
  }
  // G(tau,0) = Q_L (Db_L^-1 MI Ds_R) T_R
  for (int e = tid; e < N * N; e += kThreads) {
    const int i = e / N, j = e - i * N;
    X[(size_t)i * ld + j] = zscal(dsR[j] / dbL[i], MI[(size_t)i * ld + j]);
  }
  __syncthreads();
  zgemm<0, 0, false>(N, N, N, Lf.Q, ld, (const double2*)X, ld, Mid, ld, S.gemm);
  zgemm<0, 0, false>(N, N, N, (const double2*)Mid, ld, R.T, ld, Gt0, ld, S.gemm);
  // G(0,tau) = -T_L^H (Ds_L MI Db_R^-1) Q_R^H
  for (int e = tid; e < N * N; e += kThreads) {
    const int i = e / N, j = e - i * N;
    X[(size_t)i * ld + j] = zscal(-dsL[i] / dbR[j], MI[(size_t)i * ld + j]);
  }
  __syncthreads();
  zgemm<2, 0, false>(N, N, N, Lf.T, ld, (const double2*)X, ld, Mid, ld, S.gemm);
  zgemm<0, 2, false>(N, N, N, (const double2*)Mid, ld, R.Q, ld, G0t, ld, S.gemm);
  return 0;
}

// -g sum over every slice and site of eta(l): the phase of the bosonic factor
// exp(-i g sum eta) of the weight
__device__ double bosonic_phase(const Su2Dev& C, Sm& S) {
  double acc = 0.0;
  for (int e = threadIdx.x; e < C.L * C.N; e += kThreads) {
    const int t = e / C.N, x = e - t * C.N;
    acc += hs_eta(C.fields[(size_t)t * C.MV + x]);
  }
  return -C.g * block_sum(acc, S.red);
}

// the phase of e^{-S}: exp(i (ph + 2 arg det(1 + B))) (two colors)
__device__ inline double2 fresh_phase(double ph, double arg) { return zexpi(ph + 2.0 * arg); }

// Left chain into the storage slots, then G(0) into W6 (Algorithm 1, before the sweeps).
__device__ int z_fill_left(const Su2Dev& C, Sm& S, double& logabs, double& arg) {
  const int nst = C.L / C.nw;
  for (int j = nst - 1; j >= 0; --j) {
    const ZUdv src = (j + 1 == nst) ? z_ident(C) : z_slot(C, j + 1);
    const int dq = z_chain_step(C, j * C.nw, (j + 1) * C.nw, true, src, S);
    z_store_slot(C, j, dq);
  }
  return z_green(C, z_ident(C), z_slot(C, 0), zmat(C, 6), logabs, arg, S);
}

// ---- the sweep --------------------------------------------------------------
// V wrap: G_xy <- ph_x G_xy conj(ph_y) (ph = e^{+-V} of the slice)
__device__ void z_v_wrap(const Su2Dev& C, double2* G, const double2* ph) {
  const int N = C.N, ld = C.ld;
  for (int e = threadIdx.x; e < N * N; e += kThreads) {
    const int x = e / N, y = e - x * N;
    G[(size_t)x * ld + y] = zmul(zmul(ph[x], G[(size_t)x * ld + y]), zconj(ph[y]));
  }
  __syncthreads();
}

// T wrap: up G <- E G E^-1, down G <- E^-1 G E
__device__ void z_t_wrap(const Su2Dev& C, bool up, Sm& S) {
  const int N = C.N, ld = C.ld;
  zgemm<0, 0, false>(N, N, N, up ? C.E : C.Einv, ld, (const double2*)C.G, ld, C.Gt, ld, S.gemm);
  zgemm<0, 0, false>(N, N, N, (const double2*)C.Gt, ld, up ? C.Einv : C.E, ld, C.G, ld, S.gemm);
}

// The sites of slice tau in order (up: 0..N-1, down: N-1..0).  Per proposal:
// l' one of the other three values (index floor(3 u1)), dtheta = g (eta(l') -
// eta(l)), Delta = e^{i dtheta} - 1, r1 = 1 + Delta (1 - G~_kk),
//   R = gamma(l')/gamma(l) e^{-i dtheta} r1^2     (two colors share G~),
// accepted when u2 < min(1, |Re(P R)| / |Re P|); then P <- P R / |P R| and
// G~ <- G~ - (Delta / r1) G~[:, k] (e_k - G~[k, :]).  Rejections leave G~ and
// P unchanged, so every remaining proposal's test is evaluated in parallel and
// the first accepted one is applied.
__device__ void z_update_slice(Su2Dev& C, int tau, int dir, const Su2SweepParams& P, Sm& S) {
  const int N = C.N, ld = C.ld, tid = threadIdx.x;
  double2* G = C.G;
  const uint32_t key0 = (uint32_t)P.seed, key1 = (uint32_t)(P.seed >> 32) ^ C.chain_id;
  for (int q = tid; q < N; q += kThreads) {
    const int k = dir ? N - 1 - q : q;
    uint32_t ctr[4] = {(uint32_t)P.sweep, (uint32_t)(2 * tau + dir), (uint32_t)k, (uint32_t)(P.sweep >> 32)};
    philox4x32_10(ctr, key0, key1);
    const double u1 = uniform53(ctr[0], ctr[1]);
    S.u2[q] = uniform53(ctr[2], ctr[3]);
    const int f = S.fsl[k];
    const int fn = propose_field(2, f, u1);
    const double dth = C.g * (hs_eta(fn) - hs_eta(f));
    const double2 e = zexpi(dth);
    S.delta[q] = make_double2(e.x - 1.0, e.y);
    S.gr[q] = zscal(hs_gamma(fn) / hs_gamma(f), zconj(e));
    S.fn[q] = (int8_t)fn;
  }
  for (int x = tid; x < N; x += kThreads) S.d[x] = G[(size_t)x * ld + x];
  __syncthreads();
  int pos = 0;
  int64_t nacc = 0;
  while (pos < N) {
    if (tid == 0) *S.first = N;
    __syncthreads();
    const double2 Pc = *S.P;
    for (int q = pos + tid; q < N; q += kThreads) {
      const int k = dir ? N - 1 - q : q;
      const double2 r1 = zadd(make_double2(1.0, 0.0), zmul(S.delta[q], zsub(make_double2(1.0, 0.0), S.d[k])));
      const double2 R = zmul(S.gr[q], zmul(r1, r1));
      const double ratio = fabs(zmul(Pc, R).x) / fabs(Pc.x);
      if (S.u2[q] < (ratio < 1.0 ? ratio : 1.0)) {
        atomicMin(S.first, q);
        break;
      }
    }
    __syncthreads();
    const int first = *S.first;
    if (first >= N) break;
    const int k = dir ? N - 1 - first : first;
    const double2 r1 = zadd(make_double2(1.0, 0.0), zmul(S.delta[first], zsub(make_double2(1.0, 0.0), S.d[k])));
    const double2 coef = zdiv(S.delta[first], r1);
    for (int x = tid; x < N; x += kThreads) {
      S.col[x] = G[(size_t)x * ld + k];
      const double2 gkx = G[(size_t)k * ld + x];
      S.row[x] = make_double2((x == k ? 1.0 : 0.0) - gkx.x, -gkx.y);
    }
    __syncthreads();
    if (tid == 0) {
      const double2 R = zmul(S.gr[first], zmul(r1, r1));
      const double2 PR = zmul(Pc, R);
      *S.P = zscal(1.0 / zabs(PR), PR);
      S.fsl[k] = S.fn[first];
    }
    for (int e = tid; e < N * N; e += kThreads) {
      const int x = e / N, y = e - x * N;
      double2* gp = G + (size_t)x * ld + y;
      *gp = zsub(*gp, zmul(zmul(coef, S.col[x]), S.row[y]));
    }
    for (int x = tid; x < N; x += kThreads) S.d[x] = zsub(S.d[x], zmul(zmul(coef, S.col[x]), S.row[x]));
    ++nacc;
    pos = first + 1;
    __syncthreads();
  }
  if (tid == 0) {
    C.proposals += N;
    C.accepted += nacc;
  }
}

// Bond wraps: up G~ <- X_b G~ X_b^-1 (the bond's factor acts), down the inverse.
__device__ void z_bond_wrap(const Su2Dev& C, int b, int s, bool up) {
  const double a = C.a0 * (double)s;
  if (up) {
    bond_rows(C.N, C.ld, C.G, C.bi[b], C.bj[b], a);
    bond_cols(C.N, C.ld, C.G, C.bi[b], C.bj[b], -a);
  } else {
    bond_rows(C.N, C.ld, C.G, C.bi[b], C.bj[b], -a);
    bond_cols(C.N, C.ld, C.G, C.bi[b], C.bj[b], a);
  }
}

// Change of the bond spins' log weight when s_b of slice tau flips: the
// transverse field between neighbouring slices (periodic in tau) contributes
// log cosh(dtau h) for equal and log sinh(dtau h) for opposite spins, and each
// J pair (b, b') of the slice dtau J s_b s_b'.
__device__ double bond_dlogw(const Su2Dev& C, int tau, int b, const int8_t* fsl) {
  const int s = fsl[C.N + b];
  double dl = 0.0;
  if (C.L > 1) {
    const int tp = (tau - 2 + C.L) % C.L, tn = tau % C.L;   // 0-based neighbours of slice tau - 1
    const int nbs[2] = {C.fields[(size_t)tp * C.MV + C.N + b], C.fields[(size_t)tn * C.MV + C.N + b]};
    for (int q = 0; q < 2; ++q) {
      const double before = (s == nbs[q]) ? C.lch : C.lsh;
      const double after = (-s == nbs[q]) ? C.lch : C.lsh;
      dl += after - before;
    }
  }
  double js = 0.0;
  for (int e = C.nbr_off[b]; e < C.nbr_off[b + 1]; ++e) js += (double)fsl[C.N + C.nbr[e]];
  dl += -2.0 * C.dJ * (double)s * js;
  return dl;
}

// One bond proposal (the flip s_b -> -s_b) at the G~ its factor sees.  With
// delta = X(-2a) - 1 on the block P = (i, j), a = -dtau xi s_b, and
// S = 1 + delta (1 - G~)_PP (2 x 2):
//   R = det(S)^2 exp(dlogw)   (two colors, the spins' own weight),
// accepted when u2 < min(1, |Re(P R)| / |Re P|) (u2 from the Philox counter of
// vertex N + b); then G~ <- G~ - G~_:P S^-1 delta (1 - G~)_P: (Woodbury).
__device__ void z_bond_update(Su2Dev& C, int tau, int dir, int b, const Su2SweepParams& P, Sm& S) {
  const int N = C.N, ld = C.ld, tid = threadIdx.x;
  double2* G = C.G;
  const uint32_t key0 = (uint32_t)P.seed, key1 = (uint32_t)(P.seed >> 32) ^ C.chain_id;
  uint32_t ctr[4] = {(uint32_t)P.sweep, (uint32_t)(2 * tau + dir), (uint32_t)(N + b), (uint32_t)(P.sweep >> 32)};
  philox4x32_10(ctr, key0, key1);
  const double u2 = uniform53(ctr[2], ctr[3]);
  const int s = S.fsl[N + b];
  const double a = C.a0 * (double)s;
  const double d0 = cosh(2.0 * a) - 1.0, d1 = -sinh(2.0 * a);
  const int i = C.bi[b], j = C.bj[b];
  const double2 gii = G[(size_t)i * ld + i], gij = G[(size_t)i * ld + j];
  const double2 gji = G[(size_t)j * ld + i], gjj = G[(size_t)j * ld + j];
  const double2 h00 = make_double2(1.0 - gii.x, -gii.y), h01 = make_double2(-gij.x, -gij.y);
  const double2 h10 = make_double2(-gji.x, -gji.y), h11 = make_double2(1.0 - gjj.x, -gjj.y);
  const double2 S00 = zadd(make_double2(1.0, 0.0), zadd(zscal(d0, h00), zscal(d1, h10)));
  const double2 S01 = zadd(zscal(d0, h01), zscal(d1, h11));
  const double2 S10 = zadd(zscal(d1, h00), zscal(d0, h10));
  const double2 S11 = zadd(make_double2(1.0, 0.0), zadd(zscal(d1, h01), zscal(d0, h11)));
  const double2 det = zsub(zmul(S00, S11), zmul(S01, S10));
  const double2 R = zscal(exp(bond_dlogw(C, tau, b, S.fsl)), zmul(det, det));
  const double2 Pc = *S.P;
  const double ratio = fabs(zmul(Pc, R).x) / fabs(Pc.x);
  const bool accept = zabs(det) > 0.0 && u2 < (ratio < 1.0 ? ratio : 1.0);
  __syncthreads();
  if (tid == 0) C.proposals += 1;
  if (!accept) return;
  // W = S^-1 delta (2 x 2)
  const double2 idet = zdiv(make_double2(1.0, 0.0), det);
  const double2 I00 = zmul(S11, idet), I01 = zscal(-1.0, zmul(S01, idet));
  const double2 I10 = zscal(-1.0, zmul(S10, idet)), I11 = zmul(S00, idet);
  const double2 W00 = zadd(zscal(d0, I00), zscal(d1, I01)), W01 = zadd(zscal(d1, I00), zscal(d0, I01));
  const double2 W10 = zadd(zscal(d0, I10), zscal(d1, I11)), W11 = zadd(zscal(d1, I10), zscal(d0, I11));
  double2* c0 = S.col;    // G~[:, i]
  double2* c1 = S.hv;     // G~[:, j]
  double2* r0 = S.row;    // e_i - G~[i, :]
  double2* r1 = S.delta;  // e_j - G~[j, :]
  for (int x = tid; x < N; x += kThreads) {
    c0[x] = G[(size_t)x * ld + i];
    c1[x] = G[(size_t)x * ld + j];
    const double2 gi = G[(size_t)i * ld + x], gj = G[(size_t)j * ld + x];
    r0[x] = make_double2((x == i ? 1.0 : 0.0) - gi.x, -gi.y);
    r1[x] = make_double2((x == j ? 1.0 : 0.0) - gj.x, -gj.y);
  }
  __syncthreads();
  if (tid == 0) {
    const double2 PR = zmul(Pc, R);
    *S.P = zscal(1.0 / zabs(PR), PR);
    S.fsl[N + b] = (int8_t)(-s);
    C.accepted += 1;
  }
  for (int e = tid; e < N * N; e += kThreads) {
    const int x = e / N, y = e - x * N;
    const double2 t0 = zadd(zmul(W00, r0[y]), zmul(W01, r1[y]));
    const double2 t1 = zadd(zmul(W10, r0[y]), zmul(W11, r1[y]));
    double2* gp = G + (size_t)x * ld + y;
    *gp = zsub(*gp, zadd(zmul(c0[x], t0), zmul(c1[x], t1)));
  }
  __syncthreads();
}

// Stabilisation event j (Sec. 2.3): the chain extended by n_wrap slices, the
// stable G replaces the wrapped one (max and mean |dG| booked: "Precision
// Green"), and the fresh phase replaces the carried one (|dP| booked:
// "Precision Phase").  The new decomposition goes to slot j.
__device__ void z_stabilise(Su2Dev& C, int j, bool up, Sm& S) {
  const int N = C.N, ld = C.ld, nst = C.L / C.nw, nw = C.nw;
  int dq;
  ZUdv R, Lf;
  if (up) {
    const ZUdv src = (j == 1) ? z_ident(C) : z_slot(C, j - 1);
    dq = z_chain_step(C, (j - 1) * nw, j * nw, false, src, S);
    R = z_work(C, dq);
    Lf = (j == nst) ? z_ident(C) : z_slot(C, j);
  } else {
    const ZUdv src = (j + 1 == nst) ? z_ident(C) : z_slot(C, j + 1);
    dq = z_chain_step(C, j * nw, (j + 1) * nw, true, src, S);
    Lf = z_work(C, dq);
    R = (j == 0) ? z_ident(C) : z_slot(C, j);
  }
  double2* Gf = zmat(C, 6);
  double la = 0.0, ar = 0.0;
  const int bad = z_green(C, R, Lf, Gf, la, ar, S);
  if (bad) {
    if (threadIdx.x == 0) C.error |= 1;
    z_store_slot(C, j, dq);
    return;
  }
  double mx = 0.0, sm = 0.0;
  for (int e = threadIdx.x; e < N * N; e += kThreads) {
    const int x = e / N, y = e - x * N;
    const double2 gf = Gf[(size_t)x * ld + y];
    const double dg = zabs(zsub(gf, C.G[(size_t)x * ld + y]));
    mx = fmax(mx, dg);
    sm += dg;
    C.G[(size_t)x * ld + y] = gf;
  }
  mx = block_max(mx, S.red);
  sm = block_sum(sm, S.red);
  const double ph = bosonic_phase(C, S);
  if (threadIdx.x == 0) {
    const double2 Pf = fresh_phase(ph, ar);
    C.phase_max = fmax(C.phase_max, zabs(zsub(*S.P, Pf)));
    *S.P = Pf;
    C.prec_sum += sm / ((double)N * N);
    C.prec_max = fmax(C.prec_max, mx);
    C.prec_events += 1;
    C.logabs = la;
    C.arg = ar;
  }
  z_store_slot(C, j, dq);
}

// Energy estimator at the current G (Sec. 6.1, both colors):
//   Kin = 2 sum_xy K_xy (delta_xy - G_yx),
//   Pot = U/2 sum_i <(n_i - 1)^2> = U/2 sum_i [2 (1 - G_ii)^2 - 2 (1 - G_ii) + 1],
//   Part = 2 sum_i (1 - G_ii),
// reweighted by sign * P / Re P (Sec. 5.1: ZS, ZP).
__device__ void z_measure(Su2Dev& C, Sm& S) {
  const int N = C.N, ld = C.ld;
  double2 kin = make_double2(0.0, 0.0), pot = kin, part = kin;
  for (int e = threadIdx.x; e < N * N; e += kThreads) {
    const int x = e / N, y = e - x * N;
    const double2 g = C.G[(size_t)y * ld + x];
    const double kxy = 2.0 * C.K[(size_t)x * ld + y];
    kin = zadd(kin, make_double2(kxy * ((x == y ? 1.0 : 0.0) - g.x), -kxy * g.y));
  }
  for (int i = threadIdx.x; i < N; i += kThreads) {
    const double2 gi = C.G[(size_t)i * ld + i];
    const double2 h = make_double2(1.0 - gi.x, -gi.y);
    const double2 q = zadd(zsub(zscal(2.0, zmul(h, h)), zscal(2.0, h)), make_double2(1.0, 0.0));
    pot = zadd(pot, zscal(0.5 * C.U, q));
    part = zadd(part, zscal(2.0, h));
  }
  kin = block_zsum(kin, S.red);
  pot = block_zsum(pot, S.red);
  part = block_zsum(part, S.red);
  // bond spins: (sum_b s_b)^2 / nb averaged over the slices
  double m2 = 0.0;
  if (C.nb > 0) {
    for (int t = threadIdx.x; t < C.L; t += kThreads) {
      double mt = 0.0;
      for (int b = 0; b < C.nb; ++b) mt += (double)C.fields[(size_t)t * C.MV + N + b];
      m2 += mt * mt / (double)C.nb;
    }
    m2 = block_sum(m2, S.red) / (double)C.L;
  }
  if (threadIdx.x == 0) {
    const double2 Pc = *S.P;
    const double sg = Pc.x >= 0.0 ? 1.0 : -1.0;
    const double2 w = zscal(sg / Pc.x, Pc);
    const double2 v[5] = {zmul(w, kin), zmul(w, pot), zmul(w, part), zmul(w, zadd(kin, pot)), zscal(m2, w)};
    for (int q = 0; q < 5; ++q) {
      C.meas[2 * q] += v[q].x;
      C.meas[2 * q + 1] += v[q].y;
    }
    C.meas_sign += sg;
    C.n_meas += 1;
  }
  __syncthreads();
}

__device__ inline void load_slice(const Su2Dev& C, int tau, Sm& S) {
  for (int x = threadIdx.x; x < C.MV; x += kThreads) S.fsl[x] = C.fields[(size_t)(tau - 1) * C.MV + x];
  __syncthreads();
}
__device__ inline void store_slice(const Su2Dev& C, int tau, Sm& S) {
  for (int x = threadIdx.x; x < C.MV; x += kThreads) C.fields[(size_t)(tau - 1) * C.MV + x] = S.fsl[x];
  __syncthreads();
}

__global__ void __launch_bounds__(kThreads) su2_sweep_kernel(Su2Dev* chains, Su2SweepParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Su2Dev& C = chains[blockIdx.x];
  if (blockIdx.x >= P.n_chains) return;
  Sm S = su2_carve(smem_raw, C.N, C.MV);
  const int L = C.L, nw = C.nw;
  if (threadIdx.x == 0) *S.P = C.P;
  __syncthreads();
  for (int tau = 1; tau <= L; ++tau) {
    load_slice(C, tau, S);
    slice_phases(C, S.fsl, +1.0, S.ph);
    z_v_wrap(C, C.G, S.ph);
    z_update_slice(C, tau, 0, P, S);
    for (int b = C.nb - 1; b >= 0; --b) {
      z_bond_wrap(C, b, S.fsl[C.N + b], true);
      z_bond_update(C, tau, 0, b, P, S);
    }
    store_slice(C, tau, S);
    z_t_wrap(C, true, S);
    if (tau % nw == 0) z_stabilise(C, tau / nw, true, S);
    if (P.measure && tau >= P.meas_first && tau <= P.meas_last) z_measure(C, S);
  }
  for (int tau = L; tau >= 1; --tau) {
    load_slice(C, tau, S);
    z_t_wrap(C, false, S);
    for (int b = 0; b < C.nb; ++b) {
      z_bond_update(C, tau, 1, b, P, S);
      z_bond_wrap(C, b, S.fsl[C.N + b], false);
    }
    z_update_slice(C, tau, 1, P, S);
    store_slice(C, tau, S);
    slice_phases(C, S.fsl, -1.0, S.ph);
    z_v_wrap(C, C.G, S.ph);
    if ((tau - 1) % nw == 0) z_stabilise(C, (tau - 1) / nw, false, S);
    if (P.measure && tau - 1 >= P.meas_first && tau - 1 <= P.meas_last) z_measure(C, S);
  }
  if (threadIdx.x == 0) {
    C.P = *S.P;
    C.sweep_sign_sum += (S.P->x >= 0.0) ? 1.0 : -1.0;
  }
}

// mode 0: left chain, G(0) into the working G, log|det|, arg and the phase;
// mode 1: the same chain recomputation for chain `only`, G(0) into out
// ([N][N] complex), log|det| and arg booked, the working G and P untouched.
__global__ void __launch_bounds__(kThreads) su2_fresh_kernel(Su2Dev* chains, int n_chains, int mode, int only,
                                                            double2* out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int c = blockIdx.x;
  if (c >= n_chains || (mode == 1 && c != only)) return;
  Su2Dev& C = chains[c];
  Sm S = su2_carve(smem_raw, C.N, C.MV);
  double la = 0.0, ar = 0.0;
  if (z_fill_left(C, S, la, ar)) {
    if (threadIdx.x == 0) C.error |= 1;
    return;
  }
  const int N = C.N, ld = C.ld;
  const double2* Gf = zmat(C, 6);
  const double ph = bosonic_phase(C, S);
  for (int e = threadIdx.x; e < N * N; e += kThreads) {
    const int x = e / N, y = e - x * N;
    if (mode == 0)
      C.G[(size_t)x * ld + y] = Gf[(size_t)x * ld + y];
    else
      out[e] = Gf[(size_t)x * ld + y];
  }
  if (threadIdx.x == 0) {
    C.logabs = la;
    C.arg = ar;
    if (mode == 0) C.P = fresh_phase(ph, ar);
  }
}

// Equal-time correlation functions of each chain's current configuration from
// its working G(0) (the paper's SpinZ, Den, SpinXY and Green observables,
// collected per pair class as Obser_Latt collects them per displacement).  Both
// colors see the same G, so with X_xy = (delta_xy - G_yx) G_xy and
// rho_x = 2 (1 - G_xx), Wick's theorem gives per configuration
//   <S^z_x S^z_y> = X_xy / 2, <n_x n_y> = rho_x rho_y + 2 X_xy,
//   <S^+_x S^-_y> = X_xy,     sum_s <c^+_xs c_ys> = 2 (delta_xy - G_yx).
// One CTA per chain; thread c sums class c's pairs (CSR: pairs[off[c] ..
// off[c+1]), each x N + y) in their listed order.  out: [n_chains][max_cls][4]
// complex.
__global__ void su2_corr_kernel(const Su2Dev* chains, int n_chains, const int* const* off, const int* const* pairs,
                                const int* ncls, int max_cls, double2* out) {
  const int c = blockIdx.x;
  if (c >= n_chains) return;
  const Su2Dev& C = chains[c];
  const int N = C.N, ld = C.ld, nc = ncls[c];
  const int* o = off[c];
  const int* pr = pairs[c];
  for (int k = threadIdx.x; k < max_cls; k += blockDim.x) {
    double2 v[4];
    for (int q = 0; q < 4; ++q) v[q] = make_double2(0.0, 0.0);
    if (k < nc)
      for (int e = o[k]; e < o[k + 1]; ++e) {
        const int x = pr[e] / N, y = pr[e] - x * N;
        const double2 gyx = C.G[(size_t)y * ld + x], gxy = C.G[(size_t)x * ld + y];
        const double2 gxx = C.G[(size_t)x * ld + x], gyy = C.G[(size_t)y * ld + y];
        const double2 h = make_double2((x == y ? 1.0 : 0.0) - gyx.x, -gyx.y);
        const double2 X = zmul(h, gxy);
        const double2 rx = make_double2(2.0 * (1.0 - gxx.x), -2.0 * gxx.y);
        const double2 ry = make_double2(2.0 * (1.0 - gyy.x), -2.0 * gyy.y);
        v[0] = zadd(v[0], zscal(0.5, X));
        v[1] = zadd(v[1], zadd(zmul(rx, ry), zscal(2.0, X)));
        v[2] = zadd(v[2], X);
        v[3] = zadd(v[3], zscal(2.0, h));
      }
    for (int q = 0; q < 4; ++q) out[((size_t)c * max_cls + k) * 4 + q] = v[q];
  }
}

// The time-displaced measurement of each chain's current configuration (the
// tau_m step after a sweep, Sec. 2.4 / Algorithm 1, on the stored left chain):
// starting from the stable G(0) = (1 + B(beta,0))^-1,
//   G(tau,0) = B_tau G(tau-1,0),  G(0,tau) = G(0,tau-1) B_tau^-1,
// and at every tau = j n_wrap both are recomputed from the right chain B(tau,0)
// (built in place of the stored left chain's slot j, which is no longer needed)
// and the left chain B(beta,tau)^H; the largest and the mean |wrapped - fresh|
// entry over both is "Precision tau".  Per tau: a(tau) = sum_x G(tau,0)_xx.
// The stored left chain is rebuilt at the end, so the chain continues as it
// was; its working G is untouched.  only >= 0: that chain alone, and its
// G(n_tau,0), G(0,n_tau) ([N][N] complex) into gt0 / g0t.
__global__ void __launch_bounds__(kThreads) su2_tau_kernel(Su2Dev* chains, int n_chains, int only, int n_tau,
                                                           double2* out_a, double* out_prec, double2* gt0,
                                                           double2* g0t) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int c = blockIdx.x;
  if (c >= n_chains || (only >= 0 && c != only)) return;
  Su2Dev& C = chains[c];
  Sm S = su2_carve(smem_raw, C.N, C.MV);
  const int N = C.N, ld = C.ld, nw = C.nw, nst = C.L / nw;
  double2* Gt0 = zmat(C, 8);
  double2* G0t = zmat(C, 9);
  double2* Ft0 = zmat(C, 10);
  double2* F0t = zmat(C, 11);
  double la = 0.0, ar = 0.0;
  int bad = z_green(C, z_ident(C), z_slot(C, 0), zmat(C, 6), la, ar, S);
  const double2* G00 = zmat(C, 6);
  for (int e = threadIdx.x; e < N * N; e += kThreads) {
    const int x = e / N, y = e - x * N;
    const double2 g = G00[(size_t)x * ld + y];
    Gt0[(size_t)x * ld + y] = g;
    G0t[(size_t)x * ld + y] = make_double2(g.x - (x == y ? 1.0 : 0.0), g.y);
  }
  __syncthreads();
  double pmax = 0.0, psum = 0.0;
  int nev = 0;
  for (int tau = 0; tau <= n_tau && !bad; ++tau) {
    if (tau > 0) {
      const int8_t* f = C.fields + (size_t)(tau - 1) * C.MV;
      double2* W = zmat(C, 0);
      // G(tau,0) = E X_0 .. X_{nb-1} e^{V} G(tau-1,0)
      slice_phases(C, f, +1.0, S.ph);
      for (int e = threadIdx.x; e < N * N; e += kThreads) {
        const int x = e / N, y = e - x * N;
        Gt0[(size_t)x * ld + y] = zmul(S.ph[x], Gt0[(size_t)x * ld + y]);
      }
      __syncthreads();
      for (int b = C.nb - 1; b >= 0; --b) bond_rows(N, ld, Gt0, C.bi[b], C.bj[b], C.a0 * f[N + b]);
      zgemm<0, 0, false>(N, N, N, C.E, ld, (const double2*)Gt0, ld, W, ld, S.gemm);
      zcopy(N, ld, W, Gt0);
      // G(0,tau) = G(0,tau-1) e^{-V} X_{nb-1}^-1 .. X_0^-1 E^-1
      slice_phases(C, f, -1.0, S.ph);
      for (int e = threadIdx.x; e < N * N; e += kThreads) {
        const int x = e / N, y = e - x * N;
        G0t[(size_t)x * ld + y] = zmul(G0t[(size_t)x * ld + y], S.ph[y]);
      }
      __syncthreads();
      for (int b = C.nb - 1; b >= 0; --b) bond_cols(N, ld, G0t, C.bi[b], C.bj[b], -C.a0 * f[N + b]);
      zgemm<0, 0, false>(N, N, N, (const double2*)G0t, ld, C.Einv, ld, W, ld, S.gemm);
      zcopy(N, ld, W, G0t);
      if (tau % nw == 0) {
        const int j = tau / nw;
        const ZUdv src = (j == 1) ? z_ident(C) : z_slot(C, j - 1);
        const int dq = z_chain_step(C, (j - 1) * nw, j * nw, false, src, S);
        const ZUdv Lf = (j == nst) ? z_ident(C) : z_slot(C, j);
        bad = z_displaced(C, z_work(C, dq), Lf, Ft0, F0t, S);
        if (bad) break;
        double mx = 0.0, sm = 0.0;
        for (int e = threadIdx.x; e < N * N; e += kThreads) {
          const int x = e / N, y = e - x * N;
          const size_t q = (size_t)x * ld + y;
          const double d1 = zabs(zsub(Gt0[q], Ft0[q])), d2 = zabs(zsub(G0t[q], F0t[q]));
          mx = fmax(mx, fmax(d1, d2));
          sm += d1 + d2;
          Gt0[q] = Ft0[q];
          G0t[q] = F0t[q];
        }
        mx = block_max(mx, S.red);
        sm = block_sum(sm, S.red);
        pmax = fmax(pmax, mx);
        psum += sm / (2.0 * N * N);
        ++nev;
        z_store_slot(C, j, dq);  // the right chain B(tau,0) takes slot j
      }
    }
    double2 a = make_double2(0.0, 0.0);
    for (int x = threadIdx.x; x < N; x += kThreads) a = zadd(a, Gt0[(size_t)x * ld + x]);
    a = block_zsum(a, S.red);
    if (threadIdx.x == 0 && out_a) out_a[(size_t)c * (n_tau + 1) + tau] = a;
  }
  if (only >= 0 && !bad) {
    for (int e = threadIdx.x; e < N * N; e += kThreads) {
      const int x = e / N, y = e - x * N;
      gt0[e] = Gt0[(size_t)x * ld + y];
      g0t[e] = G0t[(size_t)x * ld + y];
    }
  }
  // the stored left chain again, for the next sweep
  if (z_fill_left(C, S, la, ar)) bad = 1;
  if (threadIdx.x == 0) {
    if (bad) C.error |= 1;
    if (out_prec) {
      out_prec[2 * c] = nev ? psum / nev : 0.0;
      out_prec[2 * c + 1] = pmax;
    }
  }
}

__global__ void su2_copy_green_kernel(Su2Dev* chains, int chain, double2* out) {
  const Su2Dev& C = chains[chain];
  const int N = C.N;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < N * N; e += gridDim.x * blockDim.x) {
    const int x = e / N, y = e - x * N;
    out[e] = C.G[(size_t)x * C.ld + y];
  }
}

// Four-valued fields i.i.d. uniform over (-2, -1, 1, 2) and bond spins i.i.d.
// +-1 from Philox (counter (0xFFFFFFFF, tau, vertex, 0xFFFFFFFF), key
// (seed_lo, seed_hi ^ chain); vertex x for site x, N + b for bond b).
__global__ void su2_init_fields_kernel(Su2Dev* chains, int n_chains, uint64_t seed) {
  const int c = blockIdx.x;
  if (c >= n_chains) return;
  const Su2Dev& C = chains[c];
  for (int e = threadIdx.x; e < C.L * C.MV; e += blockDim.x) {
    const int t = e / C.MV, k = e - t * C.MV;
    uint32_t ctr[4] = {0xFFFFFFFFu, (uint32_t)(t + 1), (uint32_t)k, 0xFFFFFFFFu};
    philox4x32_10(ctr, (uint32_t)seed, (uint32_t)(seed >> 32) ^ C.chain_id);
    const double u = uniform53(ctr[0], ctr[1]);
    if (k >= C.N) {
      C.fields[e] = u < 0.5 ? -1 : 1;
    } else {
      int idx = (int)floor(4.0 * u);
      idx = idx > 3 ? 3 : idx;
      const int8_t vals[4] = {-2, -1, 1, 2};
      C.fields[e] = vals[idx];
    }
  }
}

__global__ void su2_reset_stats_kernel(Su2Dev* chains, int n_chains, int clear_meas) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_chains) return;
  Su2Dev& C = chains[c];
  C.prec_sum = C.prec_max = C.phase_max = 0.0;
  C.prec_events = C.proposals = C.accepted = 0;
  C.sweep_sign_sum = 0.0;
  C.error = 0;
  if (clear_meas) {
    for (int q = 0; q < 10; ++q) C.meas[q] = 0.0;
    C.meas_sign = 0.0;
    C.n_meas = 0;
  }
}

}  // namespace

size_t su2_smem_bytes(int maxN, int maxMV) { return su2_smem_layout(maxN, maxMV); }

static cudaError_t su2_set_smem(const void* fn, size_t bytes) {
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t su2_launch_init_fields(Su2Dev* chains, int n_chains, uint64_t seed, cudaStream_t st) {
  su2_init_fields_kernel<<<n_chains, kThreads, 0, st>>>(chains, n_chains, seed);
  return cudaGetLastError();
}

cudaError_t su2_launch_fresh(Su2Dev* chains, int n_chains, int mode, int only, double2* out, size_t smem,
                             cudaStream_t st) {
  cudaError_t e = su2_set_smem((const void*)su2_fresh_kernel, smem);
  if (e != cudaSuccess) return e;
  su2_fresh_kernel<<<n_chains, kThreads, smem, st>>>(chains, n_chains, mode, only, out);
  return cudaGetLastError();
}

cudaError_t su2_launch_sweep(Su2Dev* chains, const Su2SweepParams& p, size_t smem, cudaStream_t st) {
  cudaError_t e = su2_set_smem((const void*)su2_sweep_kernel, smem);
  if (e != cudaSuccess) return e;
  su2_sweep_kernel<<<p.n_chains, kThreads, smem, st>>>(chains, p);
  return cudaGetLastError();
}

cudaError_t su2_launch_copy_green(Su2Dev* chains, int chain, double2* out, cudaStream_t st) {
  su2_copy_green_kernel<<<16, kThreads, 0, st>>>(chains, chain, out);
  return cudaGetLastError();
}

cudaError_t su2_launch_corr(const Su2Dev* chains, int n_chains, const int* const* off, const int* const* pairs,
                            const int* ncls, int max_cls, double2* out, cudaStream_t st) {
  su2_corr_kernel<<<n_chains, 128, 0, st>>>(chains, n_chains, off, pairs, ncls, max_cls, out);
  return cudaGetLastError();
}

cudaError_t su2_launch_tau(Su2Dev* chains, int n_chains, int only, int n_tau, double2* out_a, double* out_prec,
                           double2* gt0, double2* g0t, size_t smem, cudaStream_t st) {
  cudaError_t e = su2_set_smem((const void*)su2_tau_kernel, smem);
  if (e != cudaSuccess) return e;
  su2_tau_kernel<<<n_chains, kThreads, smem, st>>>(chains, n_chains, only, n_tau, out_a, out_prec, gt0, g0t);
  return cudaGetLastError();
}

cudaError_t su2_launch_reset_stats(Su2Dev* chains, int n_chains, int clear_meas, cudaStream_t st) {
  su2_reset_stats_kernel<<<(n_chains + 127) / 128, 128, 0, st>>>(chains, n_chains, clear_meas);
  return cudaGetLastError();
}

}  // namespace dqmc
