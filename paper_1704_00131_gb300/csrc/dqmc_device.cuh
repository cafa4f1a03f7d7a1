// GB300 (sm_103a) kernels of the BSS/DQMC sweep.
//
// Work decomposition: one thread-block cluster per Markov chain, one CTA per
// flavor (spin up / spin down of the spin-z decoupling).  The flavors are
// independent except in the acceptance ratio R = gamma * prod_s R_s, which the
// CTAs exchange through distributed shared memory; every other step (wraps,
// delayed updates, the FP64 QR/UDV stabilisation, the stable recompute of G)
// runs in the flavor's own CTA.
//
// Precision: the working Green function, the wraps and the delayed updates are
// templated on `Real` (double for the plain FP64 path, float for the mixed
// path); the stabilisation chain (B-products, pivoted QR, T update, the stable
// (1 + UDV)^-1 and log|det|) is always FP64.
//
// Method (ALF 1.0 documentation, arXiv:1704.00131):
//   B_tau = exp(-dtau K) exp(V_tau)                       Sec. 2.1, Eq. of B_tau
//   G(tau) = (1 + B(tau,0) B(beta,tau))^-1               Eq. Green_eq
//   sequential single-field updates, Metropolis         Sec. 2.2.1
//   QR-stabilised chain every n_wrap slices             Sec. 2.3, Eq. green_stable
//   sweep: tau = 1..L up, L..1 down                     Algorithm 1, Sec. 2.4
#pragma once
//
// This header holds the device code shared by the kernel translation units:
// the per-precision sweep units (dqmc_sweep_fp64.cu, dqmc_sweep_fp32.cu,
// dqmc_sweep_mixed.cu) instantiate the sweep and fresh-G kernels for one
// working precision each, so that nvcc compiles them in parallel;
// dqmc_kernels.cu holds the precision-independent kernels and the dispatch.
#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <type_traits>

#include "../../include/dqmc.h"
#include "dqmc_internal.h"

// DQMC_WITH_UMMA: 1 compiles the tensor-core product path into the float-pair
// kernels (the unit of DQMC_PREC_MIXED_TC), 0 leaves it out (the unit of
// DQMC_PREC_MIXED, whose kernels then keep their registers for the SIMT tiles).
#ifndef DQMC_WITH_UMMA
#define DQMC_WITH_UMMA 1
#endif

namespace cg = cooperative_groups;

namespace dqmc {
// Internal linkage: every translation unit that includes this header gets its
// own copy of the device code it instantiates.
namespace {

// --------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): the counter-based generator that
// draws the proposal (u1) and acceptance (u2) uniforms of every proposal.
// --------------------------------------------------------------------------
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
    const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
  }
}

__device__ __forceinline__ double uniform53(uint32_t hi, uint32_t lo) {
  const uint64_t w = ((uint64_t)hi << 32) | lo;
  return (double)(w >> 11) * 0x1.0p-53;
}

// Sub-phase cycle counter: thread 0 adds the cycles since *t0 to acc[q].
__device__ __forceinline__ void tick(long long* acc, int q, long long& t0) {
  const long long t1 = clock64();
  if (acc && threadIdx.x == 0) acc[q] += t1 - t0;
  t0 = t1;
}

// --------------------------------------------------------------------------
// Field couplings: Ising (type 1) c(s) = lambda s; four-valued HS (type 2)
// c(l) = g eta(l) with weight gamma(l) (Sec. 2.1, the discrete HS transform).
// --------------------------------------------------------------------------
__device__ __forceinline__ double hs_eta(int l) {
  const double a = sqrt(2.0 * (3.0 - sqrt(6.0))), b = sqrt(2.0 * (3.0 + sqrt(6.0)));
  return l == 1 ? a : l == -1 ? -a : l == 2 ? b : -b;
}
__device__ __forceinline__ double hs_gamma(int l) {
  return (l == 1 || l == -1) ? 1.0 + sqrt(6.0) / 3.0 : 1.0 - sqrt(6.0) / 3.0;
}
__device__ __forceinline__ double coupling(int ft, double cscale, int f) {
  return ft == 1 ? cscale * (double)f : cscale * hs_eta(f);
}
__device__ __forceinline__ double field_weight(int ft, int f) { return ft == 1 ? 1.0 : hs_gamma(f); }
// Proposal: Ising flips; HS picks one of the three other values of
// (-2,-1,1,2), in ascending order, with index floor(3 u1).
__device__ __forceinline__ int propose_field(int ft, int f, double u1) {
  if (ft == 1) return -f;
  int idx = (int)floor(3.0 * u1);
  idx = idx > 2 ? 2 : idx;
  const int vals[4] = {-2, -1, 1, 2};
  int n = 0, out = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (vals[q] != f) {
      if (n == idx) out = vals[q];
      ++n;
    }
  return out;
}
__device__ __forceinline__ double coupling_dU(int ft, double dtau, double U, double cscale, int f) {
  if (ft == 1) return 0.5 * dtau * exp(0.5 * dtau * U) / sinh(cscale) * (double)f;
  return dtau / (4.0 * cscale) * hs_eta(f);
}

// --------------------------------------------------------------------------
// Block-wide reductions (deterministic order).
// --------------------------------------------------------------------------
__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = 0.0;
#pragma unroll
  for (int w = 0; w < kThreads / 32; ++w) r += red[w];
  return r;
}
__device__ __forceinline__ double block_max(double v, double* red) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = red[0];
#pragma unroll
  for (int w = 1; w < kThreads / 32; ++w) r = fmax(r, red[w]);
  return r;
}
// argmax of v over the block, ties to the lowest index; returns the index.
__device__ __forceinline__ int block_argmax(double v, int idx, double* red, int* ired) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
    if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) { red[threadIdx.x >> 5] = v; ired[threadIdx.x >> 5] = idx; }
  __syncthreads();
  double bv = red[0];
  int bi = ired[0];
#pragma unroll
  for (int w = 1; w < kThreads / 32; ++w)
    if (red[w] > bv || (red[w] == bv && ired[w] < bi)) { bv = red[w]; bi = ired[w]; }
  return bi;
}

// --------------------------------------------------------------------------
// Float-float ("double-word") numbers: x = hi + lo with |lo| <= ulp(hi)/2,
// about 48 significant bits on the FP32 pipes, which run 64x faster than FP64
// on this GPU.  Error-free transformations: TwoSum (Knuth), FastTwoSum
// (Dekker), TwoProd with an FMA (Joldes, Muller, Popescu, ACM TOMS 2017).
// The working Green function of the mixed path is stored in this format.
// --------------------------------------------------------------------------
struct dd {
  float hi, lo;
};

__device__ __forceinline__ dd two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ dd fast_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ dd dd_add(dd a, dd b) {
  const dd s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ dd dd_mul(dd a, dd b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  return fast_two_sum(p, e);
}
// c + a * b
__device__ __forceinline__ dd dd_fma(dd a, dd b, dd c) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  const dd s = two_sum(c.hi, p);
  return fast_two_sum(s.hi, s.lo + (c.lo + e));
}

// Arithmetic adapters of the working precision (double, float, dd).
__device__ __forceinline__ double to_d(double x) { return x; }
__device__ __forceinline__ double to_d(float x) { return (double)x; }
__device__ __forceinline__ double to_d(dd x) { return (double)x.hi + (double)x.lo; }
template <typename R>
__device__ __forceinline__ R from_d(double x);
template <>
__device__ __forceinline__ double from_d<double>(double x) { return x; }
template <>
__device__ __forceinline__ float from_d<float>(double x) { return (float)x; }
template <>
__device__ __forceinline__ dd from_d<dd>(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}
__device__ __forceinline__ double rfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ dd rfma(dd a, dd b, dd c) { return dd_fma(a, b, c); }
__device__ __forceinline__ double rmul(double a, double b) { return a * b; }
__device__ __forceinline__ float rmul(float a, float b) { return a * b; }
__device__ __forceinline__ dd rmul(dd a, dd b) { return dd_mul(a, b); }
__device__ __forceinline__ double radd(double a, double b) { return a + b; }
__device__ __forceinline__ float radd(float a, float b) { return a + b; }
__device__ __forceinline__ dd radd(dd a, dd b) { return dd_add(a, b); }
__device__ __forceinline__ double rsub(double a, double b) { return a - b; }
__device__ __forceinline__ float rsub(float a, float b) { return a - b; }
__device__ __forceinline__ dd rsub(dd a, dd b) { return dd_add(a, {-b.hi, -b.lo}); }

// --------------------------------------------------------------------------
// CTA-level dense product C = op(A) op(B), row-major, generic pointers
// (global or shared).  Output tiles of 16R x 16R (R = 3, 4, 5 outputs per
// thread and dimension; R is picked per size so that N = 144 or 400 need no
// padding), 16-deep K panels staged in shared memory.  C must not alias A or B.
// --------------------------------------------------------------------------
constexpr int kGemmMaxTile = 80;  // 16 * 5

__host__ __device__ inline int gemm_pick_r(int n) {
  int best_r = 4, best = 1 << 30;
  for (int r = 5; r >= 3; --r) {
    const int t = 16 * r;
    const int padded = ((n + t - 1) / t) * t;
    if (padded < best) { best = padded; best_r = r; }
  }
  return best_r;
}

template <typename T, bool TA, bool TB, int R, bool ACC = false>
__device__ void cta_gemm_r(int M, int Nc, int Kd, const T* __restrict__ A, int lda, const T* __restrict__ B,
                           int ldb, T* __restrict__ C, int ldc, T* sm) {
  constexpr int TT = 16 * R;
  T* As = sm;            // [16][TT]
  T* Bs = sm + 16 * TT;  // [16][TT]
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (int m0 = 0; m0 < M; m0 += TT)
    for (int n0 = 0; n0 < Nc; n0 += TT) {
      T acc[R][R];
#pragma unroll
      for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j) acc[i][j] = T(0);
      for (int k0 = 0; k0 < Kd; k0 += 16) {
#pragma unroll
        for (int e = tid; e < 16 * TT; e += kThreads) {
          int r, kk;
          if (!TA) { r = e >> 4; kk = e & 15; } else { kk = e / TT; r = e - kk * TT; }
          const int gm = m0 + r, gk = k0 + kk;
          T val = T(0);
          if (gm < M && gk < Kd) val = TA ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk];
          As[kk * TT + r] = val;
        }
#pragma unroll
        for (int e = tid; e < 16 * TT; e += kThreads) {
          int kk, c;
          if (!TB) { kk = e / TT; c = e - kk * TT; } else { c = e >> 4; kk = e & 15; }
          const int gk = k0 + kk, gn = n0 + c;
          T val = T(0);
          if (gk < Kd && gn < Nc) val = TB ? B[(size_t)gn * ldb + gk] : B[(size_t)gk * ldb + gn];
          Bs[kk * TT + c] = val;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
          T a[R], b[R];
#pragma unroll
          for (int i = 0; i < R; ++i) a[i] = As[kk * TT + ty * R + i];
#pragma unroll
          for (int j = 0; j < R; ++j) b[j] = Bs[kk * TT + tx * R + j];
#pragma unroll
          for (int i = 0; i < R; ++i)
#pragma unroll
            for (int j = 0; j < R; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
      }
#pragma unroll
      for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j) {
          const int gm = m0 + ty * R + i, gn = n0 + tx * R + j;
          if (gm < M && gn < Nc) {
            if (ACC) C[(size_t)gm * ldc + gn] += acc[i][j];
            else C[(size_t)gm * ldc + gn] = acc[i][j];
          }
        }
    }
  __syncthreads();
}

template <typename T, bool TA, bool TB>
__device__ void cta_gemm(int M, int Nc, int Kd, const T* __restrict__ A, int lda, const T* __restrict__ B,
                         int ldb, T* __restrict__ C, int ldc, T* sm) {
  const int r = gemm_pick_r(M > Nc ? M : Nc);
  if (r == 3) cta_gemm_r<T, TA, TB, 3>(M, Nc, Kd, A, lda, B, ldb, C, ldc, sm);
  else if (r == 5) cta_gemm_r<T, TA, TB, 5>(M, Nc, Kd, A, lda, B, ldb, C, ldc, sm);
  else cta_gemm_r<T, TA, TB, 4>(M, Nc, Kd, A, lda, B, ldb, C, ldc, sm);
}

// The same tiling for float-float operands: every product hi*hi is split
// exactly (TwoProd), its high part summed with TwoSum into the accumulator's
// high word, the rounding errors and the hi*lo, lo*hi cross terms gathered in
// the low word and renormalised once per output.
template <bool TA, bool TB, int R, bool ACC = false>
__device__ void cta_gemm_dd_r(int M, int Nc, int Kd, const dd* __restrict__ A, int lda, const dd* __restrict__ B,
                              int ldb, dd* __restrict__ C, int ldc, dd* sm) {
  constexpr int TT = 16 * R;
  dd* As = sm;            // [16][TT]
  dd* Bs = sm + 16 * TT;  // [16][TT]
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (int m0 = 0; m0 < M; m0 += TT)
    for (int n0 = 0; n0 < Nc; n0 += TT) {
      float ah[R][R], al[R][R];
#pragma unroll
      for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j) { ah[i][j] = 0.f; al[i][j] = 0.f; }
      for (int k0 = 0; k0 < Kd; k0 += 16) {
#pragma unroll
        for (int e = tid; e < 16 * TT; e += kThreads) {
          int r, kk;
          if (!TA) { r = e >> 4; kk = e & 15; } else { kk = e / TT; r = e - kk * TT; }
          const int gm = m0 + r, gk = k0 + kk;
          dd val = {0.f, 0.f};
          if (gm < M && gk < Kd) val = TA ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk];
          As[kk * TT + r] = val;
        }
#pragma unroll
        for (int e = tid; e < 16 * TT; e += kThreads) {
          int kk, c;
          if (!TB) { kk = e / TT; c = e - kk * TT; } else { c = e >> 4; kk = e & 15; }
          const int gk = k0 + kk, gn = n0 + c;
          dd val = {0.f, 0.f};
          if (gk < Kd && gn < Nc) val = TB ? B[(size_t)gn * ldb + gk] : B[(size_t)gk * ldb + gn];
          Bs[kk * TT + c] = val;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < 16; ++kk) {
          dd a[R], b[R];
#pragma unroll
          for (int i = 0; i < R; ++i) a[i] = As[kk * TT + ty * R + i];
#pragma unroll
          for (int j = 0; j < R; ++j) b[j] = Bs[kk * TT + tx * R + j];
#pragma unroll
          for (int i = 0; i < R; ++i)
#pragma unroll
            for (int j = 0; j < R; ++j) {
              const float p = a[i].hi * b[j].hi;
              const float pe = fmaf(a[i].hi, b[j].hi, -p);
              const float s = ah[i][j] + p;
              const float bb = s - ah[i][j];
              const float se = (ah[i][j] - (s - bb)) + (p - bb);
              ah[i][j] = s;
              float lo = al[i][j] + (se + pe);
              lo = fmaf(a[i].hi, b[j].lo, lo);
              al[i][j] = fmaf(a[i].lo, b[j].hi, lo);
            }
        }
        __syncthreads();
      }
#pragma unroll
      for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j) {
          const int gm = m0 + ty * R + i, gn = n0 + tx * R + j;
          if (gm < M && gn < Nc) {
            const dd r = fast_two_sum(ah[i][j], al[i][j]);
            C[(size_t)gm * ldc + gn] = ACC ? dd_add(C[(size_t)gm * ldc + gn], r) : r;
          }
        }
    }
  __syncthreads();
}


#include "dqmc_umma.cuh"

// tile: 3 (48 x 48 output tiles) or 4 (64 x 64); 0 picks the one with less
// padding of max(M, Nc) (the autotuner may override it per context)
template <bool TA, bool TB, bool ACC>
__device__ void gemm_dd_tiles(int M, int Nc, int Kd, const dd* A, int lda, const dd* B, int ldb, dd* C, int ldc,
                              dd* sm, int tile = 0) {
  if (tile != 3 && tile != 4) {
    const int n = M > Nc ? M : Nc;
    const int p3 = (n + 47) / 48 * 48, p4 = (n + 63) / 64 * 64;
    tile = (p3 < p4) ? 3 : 4;
  }
  if (tile == 3) cta_gemm_dd_r<TA, TB, 3, ACC>(M, Nc, Kd, A, lda, B, ldb, C, ldc, sm);
  else cta_gemm_dd_r<TA, TB, 4, ACC>(M, Nc, Kd, A, lda, B, ldb, C, ldc, sm);
}

template <typename T>
__device__ __forceinline__ void cta_copy(int N, int ld, const T* src, T* dst) {
  for (int e = threadIdx.x; e < N * N; e += kThreads) {
    const int x = e / N, y = e - x * N;
    dst[(size_t)x * ld + y] = src[(size_t)x * ld + y];
  }
  __syncthreads();
}

// --------------------------------------------------------------------------
// Shared-memory layout of the sweep kernel.
// --------------------------------------------------------------------------
struct Smem {
  double* gemm;     // kGemmRegionBytes: 2*16*kGemmMaxTile doubles of the SIMT GEMM panels (also
                    // float / float-pair), or a staging buffer of the tensor-core products
  double* v;        // [ld] slice potential / exp factors
  double* ev;       // [ld]
  double* d;        // [ld] current diagonal of the effective G
  double* hv;       // [ld] Householder vector
  double* u2;       // [MV]
  double* delta;    // [MV]
  double* gam;      // [MV]
  double* Rs;       // [2][MV] own-flavor ratios, double buffered (read by the peer CTA)
  double* Rp;       // [MV] full ratio of the position a thread found accepted
  double* xdiag;    // [ld] exchange: diagonal of G for the potential energy
  double* spare;    // [ld] scratch (the float-pair QR's list of norms to recompute)
  double* xs;       // [8]  exchange: scalars
  double* red;      // [32]
  int* ired;        // [32]
  int* qsite;       // [MV]
  int* qinv;        // [ld] position in the slice's visiting order of the vertex on site x (-1: none)
  int8_t* fnew;     // [MV]
  int8_t* fslice;   // [MV] fields of the current slice
  int* expA;        // [kExpLen(ld)] row exponents of the split tensor-core products
  int* expB;        // [kExpLen(ld)] column exponents
  double* ab;       // delayed vectors A, B [2][k][ld] when they fit in shared memory
  int flavor;       // the CTA's flavor
  double* qred;     // [8][128] partial sums of the QR trailing update
  Umma um;          // tensor-core products: barriers and TMEM slot, staging aliased with ab
  int dd_tile;      // register tile of the float-pair SIMT products (0: by padding, 3, 4)
};

// The first kSmemCounterBytes of the dynamic shared memory hold thread 0's
// cycle counters of the sweep kernel (fixed addresses, no registers).
constexpr int kSmemCounterBytes = 16 * 8;

// exponent entries per operand of the split products: rows padded to the tile height
__host__ __device__ inline int exp_len(int ld) {
  const int a = umma_pad(ld, kUmmaM), b = umma_pad(ld, kUmmaNT);
  return a > b ? a : b;
}

// Shared memory of the fresh-G, measurement and adjoint kernels.  The sweep
// kernel adds the delayed vectors at the end; with the tensor-core products
// the same region (s.ab) holds their two staging buffers, which are only live
// inside a product, never while delayed vectors are pending.
constexpr int kGemmRegionBytes =
    (2 * 16 * kGemmMaxTile * 8 > kUmmaStageBytes) ? 2 * 16 * kGemmMaxTile * 8 : kUmmaStageBytes;

__host__ __device__ inline size_t smem_bytes_for(int ld, int MV) {
  size_t b = kSmemCounterBytes;
  b += kGemmRegionBytes;
  b += 6 * (size_t)ld * 8;        // v, ev, d, hv, xdiag, spare
  b += 6 * (size_t)MV * 8;        // u2, delta, gam, Rs[2], Rp
  b += 8 * 8 + 32 * 8 + 32 * 4;   // xs, red, ired
  b += (size_t)MV * 4;            // qsite
  b += (size_t)ld * 4;            // qinv
  b += 2 * (size_t)MV + 16;       // fnew, fslice
  b = (b + 15) / 16 * 16;
  b += 8 * 128 * 8;               // qred
  b += 2 * (size_t)exp_len(ld) * 4;  // expA, expB
  b = (b + 15) / 16 * 16;
  b += 128;                       // mbarriers and the TMEM slot of the tensor-core products
  return b;
}
// Bytes of the region at s.ab (start 128-byte aligned by carve_smem): the
// delayed vectors, or the second and third staging buffers of the tensor-core
// products (the first is the GEMM region).
__host__ __device__ inline size_t smem_tail_bytes(size_t ab_bytes, bool umma) {
  const size_t st = umma ? (size_t)(kUmmaStages - 1) * kUmmaStageBytes : 0;
  return 128 + (ab_bytes > st ? ab_bytes : st);
}

__device__ inline Smem carve_smem(unsigned char* base, int ld, int MV) {
  Smem s;
  base += kSmemCounterBytes;
  double* p = reinterpret_cast<double*>(base);
  s.gemm = p; p += kGemmRegionBytes / 8;
  s.v = p; p += ld;
  s.ev = p; p += ld;
  s.d = p; p += ld;
  s.hv = p; p += ld;
  s.xdiag = p; p += ld;
  s.spare = p; p += ld;
  s.u2 = p; p += MV;
  s.delta = p; p += MV;
  s.gam = p; p += MV;
  s.Rs = p; p += 2 * MV;
  s.Rp = p; p += MV;
  s.xs = p; p += 8;
  s.red = p; p += 32;
  int* ip = reinterpret_cast<int*>(p);
  s.ired = ip; ip += 32;
  s.qsite = ip; ip += MV;
  s.qinv = ip; ip += ld;
  int8_t* bp = reinterpret_cast<int8_t*>(ip);
  s.fnew = bp; bp += MV;
  s.fslice = bp; bp += MV + 16;
  const size_t off = ((size_t)(bp - reinterpret_cast<int8_t*>(base)) + 15) / 16 * 16;
  s.qred = reinterpret_cast<double*>(base + off);
  const int le = exp_len(ld);
  s.expA = reinterpret_cast<int*>(s.qred + 8 * 128);
  s.expB = s.expA + le;
  unsigned char* q = reinterpret_cast<unsigned char*>(s.expB + le);
  q = base + (((size_t)(q - base) + 15) / 16 * 16);
  s.um.bar = reinterpret_cast<uint64_t*>(q);                 // 2 kUmmaStages mbarriers, counters
  s.um.tmem_slot = reinterpret_cast<uint32_t*>(q + 96);
  s.um.err = nullptr;
  s.um.where = nullptr;
  s.dd_tile = 0;
  s.um.limit = kUmmaWaitCycles;
  s.um.stall = 0;
  s.um.tmA = nullptr;
  s.um.tmB = nullptr;
  s.um.boff = 0;
  q += 128;
  // base is 16-byte aligned (kSmemCounterBytes past the start); align s.ab to 128
  const uintptr_t qa = (reinterpret_cast<uintptr_t>(q) + 127) & ~(uintptr_t)127;
  s.ab = reinterpret_cast<double*>(qa);
  s.um.stage0 = reinterpret_cast<unsigned char*>(s.gemm);
  s.um.stage1 = reinterpret_cast<unsigned char*>(qa);
  return s;
}

// Float-pair product of the mixed path: exact-split tensor-core products when
// the chain has digit-plane scratch, the float-pair SIMT tiles otherwise.
template <bool TA, bool TB, bool ACC>
__device__ void gemm_dd(const ChainDev& C, int s, Smem& S, int M, int Nc, int Kd, const dd* A, int lda, const dd* B,
                        int ldb, dd* Cm, int ldc, int constA = -1, int constB = -1) {
#if DQMC_WITH_UMMA
  if (C.planes[s]) {
    // constA / constB: index of a prepared constant operand (kCpEA ...), -1: split here
    const UmmaOperand cA = constA >= 0 ? UmmaOperand{(const __nv_bfloat16*)C.cpl[s][constA], C.cex[s][constA],
                                                     &C.tm_cp[s][constA]}
                                       : UmmaOperand{nullptr, nullptr, nullptr};
    const UmmaOperand cB = constB >= 0 ? UmmaOperand{(const __nv_bfloat16*)C.cpl[s][constB], C.cex[s][constB],
                                                     &C.tm_cp[s][constB]}
                                       : UmmaOperand{nullptr, nullptr, nullptr};
    gemm_umma<TA, TB, ACC>(M, Nc, Kd, A, lda, B, ldb, Cm, ldc, (__nv_bfloat16*)C.planes[s], S.expA, S.expB, S.um,
                           cA, cB);
    return;
  }
#else
  (void)constA;
  (void)constB;
#endif
  gemm_dd_tiles<TA, TB, ACC>(M, Nc, Kd, A, lda, B, ldb, Cm, ldc, reinterpret_cast<dd*>(S.gemm), S.dd_tile);
}

// Slice potential v^s_i of slice tau (1-based) from global fields.
__device__ void slice_potential_global(const ChainDev& C, int s, int tau, double* v) {
  for (int x = threadIdx.x; x < C.N; x += kThreads) v[x] = 0.0;
  __syncthreads();
  for (int k = threadIdx.x; k < C.MV; k += kThreads)
    v[C.site[k]] = C.vsign[s * C.MV + k] * coupling(C.ft, C.cscale, C.fields[(size_t)(tau - 1) * C.MV + k]);
  __syncthreads();
}

// Slice potential from the shared-memory copy of the slice's fields.
__device__ void slice_potential_smem(const ChainDev& C, int s, const int8_t* fsl, double* v) {
  for (int x = threadIdx.x; x < C.N; x += kThreads) v[x] = 0.0;
  __syncthreads();
  for (int k = threadIdx.x; k < C.MV; k += kThreads)
    v[C.site[k]] = C.vsign[s * C.MV + k] * coupling(C.ft, C.cscale, fsl[k]);
  __syncthreads();
}

// --------------------------------------------------------------------------
// FP64 stabilisation building blocks (Sec. 2.3).
// --------------------------------------------------------------------------
struct UDV {
  const double* Q;
  const double* D;
  const double* T;
  int detq;
};

__device__ inline double* wmat(const ChainDev& C, int s, int m) {
  return C.work[s] + (size_t)m * C.N * C.ld;
}
__device__ inline double* wvec(const ChainDev& C, int s, int v) {
  return C.work[s] + (size_t)kWorkMats * C.N * C.ld + (size_t)v * C.ld;
}
__device__ inline UDV ident_udv(const ChainDev& C) {
  UDV u;
  u.Q = C.ident;
  u.T = C.ident + (size_t)C.N * C.ld;
  u.D = C.ident + (size_t)2 * C.N * C.ld;
  u.detq = 1;
  return u;
}
__device__ inline double* slot_base(const ChainDev& C, int s, int j) {
  return C.slots[s] + (size_t)j * slot_stride(C.N, C.ld);
}
__device__ inline UDV slot_udv(const ChainDev& C, int s, int j) {
  UDV u;
  double* b = slot_base(C, s, j);
  u.Q = b;
  u.T = b + (size_t)C.N * C.ld;
  u.D = b + (size_t)2 * C.N * C.ld;
  u.detq = C.slot_detq[s][j];
  return u;
}

// M[k:, j] -= bk v (v^T M[k:, j]) for the columns j0 <= j < N, v = hv[k:].
// 8 row groups x 32 columns: rows are read coalesced along j; the partial dot
// products of the row groups are summed in shared memory in a fixed order.
__device__ void householder_apply(int N, int ld, double* M, int k, int j0, double bk, const double* hv,
                                  double* qred) {
  const int tid = threadIdx.x, lane = tid & 31, rg = tid >> 5;
  for (int c0 = j0; c0 < N; c0 += 128) {
    double w[4] = {0.0, 0.0, 0.0, 0.0};
    int i = k + rg;
    // four rows per iteration with all loads issued first (memory-level parallelism)
    for (; i + 24 < N; i += 32) {
      double x[4][4];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int j = c0 + lane + 32 * q;
          x[r][q] = (j < N) ? M[(size_t)(i + 8 * r) * ld + j] : 0.0;
        }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const double vi = hv[i + 8 * r];
#pragma unroll
        for (int q = 0; q < 4; ++q) w[q] = fma(vi, x[r][q], w[q]);
      }
    }
    for (; i < N; i += 8) {
      const double vi = hv[i];
      const double* row = M + (size_t)i * ld;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int j = c0 + lane + 32 * q;
        if (j < N) w[q] = fma(vi, row[j], w[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) qred[rg * 128 + lane + 32 * q] = w[q];
    __syncthreads();
    double wt[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      double t = 0.0;
#pragma unroll
      for (int r = 0; r < 8; ++r) t += qred[r * 128 + lane + 32 * q];
      wt[q] = bk * t;
    }
    i = k + rg;
    for (; i + 24 < N; i += 32) {
      double x[4][4];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int j = c0 + lane + 32 * q;
          x[r][q] = (j < N) ? M[(size_t)(i + 8 * r) * ld + j] : 0.0;
        }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const double vi = hv[i + 8 * r];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int j = c0 + lane + 32 * q;
          if (j < N) M[(size_t)(i + 8 * r) * ld + j] = x[r][q] - wt[q] * vi;
        }
      }
    }
    for (; i < N; i += 8) {
      const double vi = hv[i];
      double* row = M + (size_t)i * ld;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int j = c0 + lane + 32 * q;
        if (j < N) row[j] -= wt[q] * vi;
      }
    }
    __syncthreads();
  }
}

// Householder QR with column pivoting of M (N x N, in place): on return the
// upper triangle holds R, the strict lower triangle the Householder vectors
// (their leading entries in vk0), beta[k] the reflector coefficients,
// perm[k] the original column at position k.  Returns det(Q) = (-1)^#reflectors.
// Pivot = remaining column of largest norm (ties to the lowest index); norms
// are downdated and recomputed when cancellation sets in (LAPACK xGEQP3 rule).
__device__ int qr_pivoted(int N, int ld, double* M, double* beta, double* vk0, double* cn, double* cn0,
                          int* perm, Smem& S) {
  const int tid = threadIdx.x;
  for (int j = tid; j < N; j += kThreads) {
    double acc = 0.0;
    for (int i = 0; i < N; ++i) acc = fma(M[(size_t)i * ld + j], M[(size_t)i * ld + j], acc);
    cn[j] = sqrt(acc);
    cn0[j] = cn[j];
    perm[j] = j;
  }
  __syncthreads();
  const double tol3z = sqrt(2.220446049250313e-16);
  int detq = 1;
  for (int k = 0; k < N; ++k) {
    // pivot
    double bv = -1.0;
    int bi = N;
    for (int j = k + tid; j < N; j += kThreads)
      if (cn[j] > bv) { bv = cn[j]; bi = j; }
    int p = block_argmax(bv, bi, S.red, S.ired);
    if (p >= N) p = k;  // no finite candidate (NaN input): keep the column order
    if (p != k) {
      for (int i = tid; i < N; i += kThreads) {
        const double t = M[(size_t)i * ld + k];
        M[(size_t)i * ld + k] = M[(size_t)i * ld + p];
        M[(size_t)i * ld + p] = t;
      }
      if (tid == 0) {
        const int tp = perm[k]; perm[k] = perm[p]; perm[p] = tp;
        double t = cn[k]; cn[k] = cn[p]; cn[p] = t;
        t = cn0[k]; cn0[k] = cn0[p]; cn0[p] = t;
      }
      __syncthreads();
    }
    // reflector from column k, rows k..N-1
    double part = 0.0;
    for (int i = k + tid; i < N; i += kThreads) {
      const double x = M[(size_t)i * ld + k];
      part = fma(x, x, part);
      S.hv[i] = x;
    }
    const double xn2 = block_sum(part, S.red);
    const double xnorm = sqrt(xn2);
    const double x0 = S.hv[k];
    double bk = 0.0;
    double alpha = 0.0;
    if (xnorm > 0.0) {
      alpha = (x0 >= 0.0) ? -xnorm : xnorm;
      const double v0 = x0 - alpha;
      const double vtv = xn2 - x0 * x0 + v0 * v0;
      bk = (vtv > 0.0) ? 2.0 / vtv : 0.0;
      __syncthreads();
      if (tid == 0) S.hv[k] = v0;
      __syncthreads();
    }
    if (tid == 0) {
      beta[k] = bk;
      vk0[k] = S.hv[k];
    }
    if (bk != 0.0) detq = -detq;
    // apply H = I - bk v v^T to the trailing columns j > k
    if (bk != 0.0) householder_apply(N, ld, M, k, k + 1, bk, S.hv, S.qred);
    __syncthreads();
    if (tid == 0) M[(size_t)k * ld + k] = (xnorm > 0.0) ? alpha : x0;
    // downdate the trailing column norms
    for (int j = k + 1 + tid; j < N; j += kThreads) {
      if (cn[j] != 0.0) {
        double t = fabs(M[(size_t)k * ld + j]) / cn[j];
        t = fmax(0.0, (1.0 + t) * (1.0 - t));
        const double r = cn[j] / cn0[j];
        if (t * r * r <= tol3z) {
          double acc = 0.0;
          for (int i = k + 1; i < N; ++i) acc = fma(M[(size_t)i * ld + j], M[(size_t)i * ld + j], acc);
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

// Q = H_0 H_1 ... H_{N-1} from the reflectors left in M by qr_pivoted.
__device__ void form_q(int N, int ld, const double* M, const double* beta, const double* vk0, double* Q,
                       Smem& S) {
  const int tid = threadIdx.x;
  for (int e = tid; e < N * N; e += kThreads) {
    const int x = e / N, y = e - x * N;
    Q[(size_t)x * ld + y] = (x == y) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int k = N - 1; k >= 0; --k) {
    const double bk = beta[k];
    if (bk == 0.0) continue;
    for (int i = k + tid; i < N; i += kThreads) S.hv[i] = (i == k) ? vk0[k] : M[(size_t)i * ld + k];
    __syncthreads();
    householder_apply(N, ld, Q, k, k, bk, S.hv, S.qred);
  }
}

// One step of a UDV chain (Sec. 2.3): X = Bcal Q_src, M = X D_src, M P = Q R,
// D = |diag R|, T = D^-1 R P^T T_src.  Right chain (left == false): Bcal =
// B_t2 ... B_t1+1.  Left chain: Bcal = B_t1+1^T ... B_t2^T.  Result in
// (W2, wvec 0, W5); returns det(Q).
// One-sided Jacobi SVD (Hestenes) of M = U S V^T, N x N in place: column
// pairs of M are rotated until mutually orthogonal (|m_p . m_q| <= 1e-15
// |m_p| |m_q| for every pair, at most 60 sweeps); then S_j = |m_j|, the
// columns of M are normalised to U (e_j for a zero column) and V holds the
// product of the rotations.  One-sided Jacobi keeps the relative accuracy of
// the small singular values of a column-scaled matrix, which is what the scale
// separation of the stable G needs.  The pairs of a sweep follow the
// round-robin (circle) schedule, N/2 disjoint pairs per round, one warp per
// pair; every warp sums its dot products in the same butterfly order, so the
// result does not depend on timing.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ void svd_jacobi(int N, int ld, double* M, double* V, double* Sv) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < N * N; e += kThreads) {
    const int x = e / N, y = e - x * N;
    V[(size_t)x * ld + y] = (x == y) ? 1.0 : 0.0;
  }
  __syncthreads();
  const int n = N + (N & 1);  // players of the schedule (a dummy when N is odd)
  for (int sweep = 0; sweep < 60; ++sweep) {
    int rotated = 0;
    for (int r = 0; r < n - 1; ++r) {
      for (int k = warp; k < n / 2; k += kThreads / 32) {
        int p = (k == 0) ? n - 1 : (r + k) % (n - 1);
        int q = (k == 0) ? r : (r - k + n - 1) % (n - 1);
        if (p > q) { const int t = p; p = q; q = t; }
        if (q >= N) continue;
        double a = 0.0, b = 0.0, c = 0.0;
        for (int i = lane; i < N; i += 32) {
          const double xp = M[(size_t)i * ld + p], xq = M[(size_t)i * ld + q];
          a = fma(xp, xp, a);
          b = fma(xq, xq, b);
          c = fma(xp, xq, c);
        }
        a = warp_sum(a);
        b = warp_sum(b);
        c = warp_sum(c);
        if (c == 0.0 || fabs(c) <= 1e-15 * sqrt(a * b)) continue;
        rotated = 1;
        const double zeta = (b - a) / (2.0 * c);
        const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
        for (int i = lane; i < N; i += 32) {
          double* mp = M + (size_t)i * ld + p;
          double* mq = M + (size_t)i * ld + q;
          const double xp = *mp, xq = *mq;
          *mp = cs * xp - sn * xq;
          *mq = sn * xp + cs * xq;
          double* vp = V + (size_t)i * ld + p;
          double* vq = V + (size_t)i * ld + q;
          const double yp = *vp, yq = *vq;
          *vp = cs * yp - sn * yq;
          *vq = sn * yp + cs * yq;
        }
      }
      __syncthreads();
    }
    if (!__syncthreads_or(rotated)) break;
  }
  for (int j = tid; j < N; j += kThreads) {
    double s2 = 0.0;
    for (int i = 0; i < N; ++i) s2 = fma(M[(size_t)i * ld + j], M[(size_t)i * ld + j], s2);
    Sv[j] = sqrt(s2);
  }
  __syncthreads();
  for (int e = tid; e < N * N; e += kThreads) {
    const int x = e / N, y = e - x * N;
    const double sj = Sv[y];
    M[(size_t)x * ld + y] = (sj > 0.0) ? M[(size_t)x * ld + y] / sj : (x == y ? 1.0 : 0.0);
  }
  __syncthreads();
}

template <typename T>
__device__ int lu_factor_blk(int N, int ld, T* A, int* piv, T* tmp, double& logdet, int& sign, Smem& S);

__device__ int chain_step(const ChainDev& C, int s, int t1, int t2, bool left, UDV src, Smem& S,
                      long long* det = nullptr) {
  long long t0 = clock64();
  const int N = C.N, ld = C.ld;
  double* X = wmat(C, s, 0);
  double* Y = wmat(C, s, 1);
  cta_copy(N, ld, src.Q, X);
  const double* E = C.E[s];
  if (!left) {
    for (int t = t1 + 1; t <= t2; ++t) {
      slice_potential_global(C, s, t, S.v);
      for (int x = threadIdx.x; x < N; x += kThreads) S.ev[x] = exp(S.v[x]);
      __syncthreads();
      for (int e = threadIdx.x; e < N * N; e += kThreads) {
        const int x = e / N, y = e - x * N;
        X[(size_t)x * ld + y] *= S.ev[x];
      }
      __syncthreads();
      cta_gemm<double, false, false>(N, N, N, E, ld, X, ld, Y, ld, S.gemm);
      double* t_ = X; X = Y; Y = t_;
    }
  } else {
    for (int t = t2; t >= t1 + 1; --t) {
      cta_gemm<double, true, false>(N, N, N, E, ld, X, ld, Y, ld, S.gemm);
      slice_potential_global(C, s, t, S.v);
      for (int x = threadIdx.x; x < N; x += kThreads) S.ev[x] = exp(S.v[x]);
      __syncthreads();
      for (int e = threadIdx.x; e < N * N; e += kThreads) {
        const int x = e / N, y = e - x * N;
        Y[(size_t)x * ld + y] *= S.ev[x];
      }
      __syncthreads();
      double* t_ = X; X = Y; Y = t_;
    }
  }
  tick(det, 4, t0);
  // M = X D_src
  for (int e = threadIdx.x; e < N * N; e += kThreads) {
    const int x = e / N, y = e - x * N;
    X[(size_t)x * ld + y] *= src.D[y];
  }
  __syncthreads();
  double* Dn = wvec(C, s, 0);
  if (C.stab_svd) {
    // M = U S V^T: Q = U, D = S, T = V^T T_src, det Q from an LU of U
    double* V = Y;
    svd_jacobi(N, ld, X, V, Dn);
    double* Qn = wmat(C, s, 2);
    double* Ucp = wmat(C, s, 3);
    for (int e = threadIdx.x; e < N * N; e += kThreads) {
      const int x = e / N, y = e - x * N;
      Qn[(size_t)x * ld + y] = X[(size_t)x * ld + y];
      Ucp[(size_t)x * ld + y] = X[(size_t)x * ld + y];
    }
    __syncthreads();
    double ldu;
    int detq = 1;
    if (lu_factor_blk(N, ld, Ucp, C.iwork[s] + ld, wmat(C, s, 9), ldu, detq, S)) detq = 1;
    tick(det, 5, t0);
    cta_gemm<double, true, false>(N, N, N, V, ld, src.T, ld, wmat(C, s, 5), ld, S.gemm);
    tick(det, 6, t0);
    return detq;
  }
  double* beta = wvec(C, s, 1);
  double* vk0 = wvec(C, s, 2);
  int* perm = C.iwork[s];
  const int detq = qr_pivoted(N, ld, X, beta, vk0, wvec(C, s, 3), wvec(C, s, 4), perm, S);
  double* Qn = wmat(C, s, 2);
  form_q(N, ld, X, beta, vk0, Qn, S);
  tick(det, 5, t0);
  double* PT = wmat(C, s, 3);
  double* Rt = wmat(C, s, 4);
  for (int x = threadIdx.x; x < N; x += kThreads) Dn[x] = fabs(X[(size_t)x * ld + x]);
  __syncthreads();
  for (int e = threadIdx.x; e < N * N; e += kThreads) {
    const int x = e / N, y = e - x * N;
    PT[(size_t)x * ld + y] = src.T[(size_t)perm[x] * ld + y];
    Rt[(size_t)x * ld + y] = (y >= x && Dn[x] > 0.0) ? X[(size_t)x * ld + y] / Dn[x] : 0.0;
  }
  __syncthreads();
  cta_gemm<double, false, false>(N, N, N, Rt, ld, PT, ld, wmat(C, s, 5), ld, S.gemm);
  tick(det, 6, t0);
  return detq;
}

// LU and solves of the middle matrix, blocked, templated on double and float
// pairs.  On the mixed path they run in float pairs on the FP32 pipes: every
// row of Mid has an entry of order one (for each i either Db_R,i = 1 or
// Ds_R,i = 1, and likewise for the columns), so Mid, its LU factors and the
// solution X = Mid^-1 Db_R^-1 Q_R^T stay inside the float range; entries that
// underflow are below 1e-38 of their row and change G by less than that in
// absolute value.  Pivots are chosen on |hi + lo| in FP64 and divisions use the
// FP64 reciprocal of the pivot.
//
// Blocking: a panel of PB columns (or a block of PB rows of the right-hand
// sides) is staged in the shared GEMM buffer and finished there; everything
// beyond it is updated by one accumulate-GEMM of depth PB.  PB is the largest
// power of two <= 16 with PB (N + PB) elements fitting the buffer.
__device__ __forceinline__ double rneg(double a) { return -a; }
__device__ __forceinline__ dd rneg(dd a) { return {-a.hi, -a.lo}; }

__device__ inline int lu_block_width(int N) {
  const int cap = 2 * 16 * kGemmMaxTile;
  int pb = 16;
  while (pb > 1 && pb * (N + pb) > cap) pb >>= 1;
  return pb;
}

// C += A B (row-major, no transposes) on the register-tiled CTA products.
__device__ inline void gemm_acc(int M, int Nc, int Kd, const double* A, int lda, const double* B, int ldb, double* C,
                                int ldc, Smem& S) {
  const int r = gemm_pick_r(M > Nc ? M : Nc);
  if (r == 3) cta_gemm_r<double, false, false, 3, true>(M, Nc, Kd, A, lda, B, ldb, C, ldc, S.gemm);
  else if (r == 5) cta_gemm_r<double, false, false, 5, true>(M, Nc, Kd, A, lda, B, ldb, C, ldc, S.gemm);
  else cta_gemm_r<double, false, false, 4, true>(M, Nc, Kd, A, lda, B, ldb, C, ldc, S.gemm);
}
__device__ inline void gemm_acc(int M, int Nc, int Kd, const dd* A, int lda, const dd* B, int ldb, dd* C, int ldc,
                                Smem& S) {
  gemm_dd_tiles<false, false, true>(M, Nc, Kd, A, lda, B, ldb, C, ldc, reinterpret_cast<dd*>(S.gemm), S.dd_tile);
}

// P A = L U in place (unit L below the diagonal, rows interchanged whole);
// piv[k] = row interchanged with row k.  tmp: PB x N scratch (ld).  Returns 1 if
// a pivot column has no finite nonzero entry.
template <typename T>
__device__ int lu_factor_blk(int N, int ld, T* A, int* piv, T* tmp, double& logdet, int& sign, Smem& S) {
  const int tid = threadIdx.x;
  const int PB = lu_block_width(N);
  T* P = reinterpret_cast<T*>(S.gemm);
  double ld_ = 0.0;
  int sg = 1;
  for (int k0 = 0; k0 < N; k0 += PB) {
    const int nb = (N - k0 < PB) ? N - k0 : PB, rows = N - k0, n2 = N - k0 - nb;
    for (int e = tid; e < rows * nb; e += kThreads) {
      const int r = e / nb, q = e - r * nb;
      P[r * PB + q] = A[(size_t)(k0 + r) * ld + k0 + q];
    }
    __syncthreads();
    for (int c = 0; c < nb; ++c) {
      double bv = -1.0;
      int bi = rows;
      for (int r = c + tid; r < rows; r += kThreads) {
        const double a = fabs(to_d(P[r * PB + c]));
        if (a > bv) { bv = a; bi = r; }
      }
      const int p = block_argmax(bv, bi, S.red, S.ired);
      if (p >= rows) return 1;
      if (tid == 0) piv[k0 + c] = k0 + p;
      const double pv = to_d(P[p * PB + c]);
      if (!(pv != 0.0)) return 1;
      if (p != c) {
        for (int q = tid; q < nb; q += kThreads) {
          const T t = P[c * PB + q];
          P[c * PB + q] = P[p * PB + q];
          P[p * PB + q] = t;
        }
        sg = -sg;
      }
      __syncthreads();
      const double d = to_d(P[c * PB + c]);
      ld_ += log(fabs(d));
      if (d < 0.0) sg = -sg;
      const T dinv = from_d<T>(1.0 / d);
      for (int r = c + 1 + tid; r < rows; r += kThreads) {
        const T l = rmul(P[r * PB + c], dinv);
        P[r * PB + c] = l;
        const T ml = rneg(l);
        for (int q = c + 1; q < nb; ++q) P[r * PB + q] = rfma(ml, P[c * PB + q], P[r * PB + q]);
      }
      __syncthreads();
    }
    for (int e = tid; e < rows * nb; e += kThreads) {
      const int r = e / nb, q = e - r * nb;
      A[(size_t)(k0 + r) * ld + k0 + q] = P[r * PB + q];
    }
    // the panel's interchanges on the columns outside it (one thread per column)
    for (int j = tid; j < N; j += kThreads) {
      if (j >= k0 && j < k0 + nb) continue;
      for (int c = 0; c < nb; ++c) {
        const int p = piv[k0 + c];
        if (p != k0 + c) {
          const T t = A[(size_t)(k0 + c) * ld + j];
          A[(size_t)(k0 + c) * ld + j] = A[(size_t)p * ld + j];
          A[(size_t)p * ld + j] = t;
        }
      }
    }
    __syncthreads();
    if (n2 > 0) {
      // U12 = L11^-1 A12 column by column (L11 = P rows 0..nb-1, staging after it)
      T* U = P + PB * PB;
      for (int jj = tid; jj < n2; jj += kThreads) {
        const int j = k0 + nb + jj;
        for (int q = 0; q < nb; ++q) {
          T u = A[(size_t)(k0 + q) * ld + j];
          for (int p2 = 0; p2 < q; ++p2) u = rfma(rneg(P[q * PB + p2]), U[p2 * n2 + jj], u);
          U[q * n2 + jj] = u;
          A[(size_t)(k0 + q) * ld + j] = u;
          tmp[(size_t)q * ld + jj] = rneg(u);
        }
      }
      __syncthreads();
      // A22 -= L21 U12
      gemm_acc(rows - nb, n2, nb, A + (size_t)(k0 + nb) * ld + k0, ld, tmp, ld, A + (size_t)(k0 + nb) * ld + k0 + nb,
               ld, S);
    }
  }
  logdet = ld_;
  sign = sg;
  return 0;
}

// Solve (LU) X = B for all N columns of B, B already in interchanged row order
// (B <- X).  Blocks of PB rows are solved in shared memory, one thread per
// column; the rows beyond a block are updated by one accumulate-GEMM.  tmp: PB x N.
template <typename T>
__device__ void lu_solve_blk(int N, int ld, const T* LU, T* B, T* tmp, Smem& S) {
  const int tid = threadIdx.x;
  const int PB = lu_block_width(N);
  T* Lb = reinterpret_cast<T*>(S.gemm);  // [PB][PB] diagonal block
  T* Y = Lb + PB * PB;                   // [PB][N] block of right-hand sides
  for (int pass = 0; pass < 2; ++pass) {
    const int nblk = (N + PB - 1) / PB;
    for (int bi = 0; bi < nblk; ++bi) {
      // forward: blocks top to bottom; backward: bottom to top
      const int r0 = pass == 0 ? bi * PB : (nblk - 1 - bi) * PB;
      const int nb = (N - r0 < PB) ? N - r0 : PB;
      for (int e = tid; e < nb * nb; e += kThreads) {
        const int q = e / nb, p2 = e - q * nb;
        Lb[q * PB + p2] = LU[(size_t)(r0 + q) * ld + r0 + p2];
      }
      for (int e = tid; e < nb * N; e += kThreads) {
        const int q = e / N, j = e - q * N;
        Y[q * N + j] = B[(size_t)(r0 + q) * ld + j];
      }
      __syncthreads();
      for (int j = tid; j < N; j += kThreads) {
        if (pass == 0) {
          for (int q = 1; q < nb; ++q) {
            T y = Y[q * N + j];
            for (int p2 = 0; p2 < q; ++p2) y = rfma(rneg(Lb[q * PB + p2]), Y[p2 * N + j], y);
            Y[q * N + j] = y;
          }
        } else {
          for (int q = nb - 1; q >= 0; --q) {
            T y = Y[q * N + j];
            for (int p2 = q + 1; p2 < nb; ++p2) y = rfma(rneg(Lb[q * PB + p2]), Y[p2 * N + j], y);
            Y[q * N + j] = rmul(y, from_d<T>(1.0 / to_d(Lb[q * PB + q])));
          }
        }
        for (int q = 0; q < nb; ++q) {
          const T y = Y[q * N + j];
          B[(size_t)(r0 + q) * ld + j] = y;
          tmp[(size_t)q * ld + j] = rneg(y);
        }
      }
      __syncthreads();
      if (pass == 0 && r0 + nb < N)
        gemm_acc(N - r0 - nb, N, nb, LU + (size_t)(r0 + nb) * ld + r0, ld, tmp, ld, B + (size_t)(r0 + nb) * ld, ld, S);
      if (pass == 1 && r0 > 0) gemm_acc(r0, N, nb, LU + r0, ld, tmp, ld, B, ld, S);
    }
  }
}

// Row map of the LU row interchanges: row i of P b is row rowof[i] of b.
__device__ void lu_row_map(int N, const int* piv, int* rowof) {
  if (threadIdx.x == 0) {
    for (int i = 0; i < N; ++i) rowof[i] = i;
    for (int k = 0; k < N; ++k) {
      const int p = piv[k];
      const int t = rowof[k]; rowof[k] = rowof[p]; rowof[p] = t;
    }
  }
  __syncthreads();
}

// Stable G from a right chain R (B(tau,0) = Q_R D_R T_R) and a left chain Lf
// (B(beta,tau)^T = Q_L D_L T_L) by scale separation, D = Db Ds with
// Db = max(D,1), Ds = min(D,1):
//   Mid = Db_R^-1 Q_R^T Q_L Db_L^-1 + Ds_R (T_R T_L^T) Ds_L
//   G   = Q_L Db_L^-1 Mid^-1 Db_R^-1 Q_R^T
//   log|det G^-1| = sum log Db_R + sum log Db_L + log|det Mid|.
// Uses W0, W1; the result goes to Gout.  Returns nonzero if Mid is singular.
__device__ int green_from_udv(const ChainDev& C, int s, UDV R, UDV Lf, double* Gout, double& logdet,
                              int& sign, Smem& S) {
  const int N = C.N, ld = C.ld;
  double* W0 = wmat(C, s, 0);
  double* W1 = wmat(C, s, 1);
  cta_gemm<double, true, false>(N, N, N, R.Q, ld, Lf.Q, ld, W0, ld, S.gemm);
  cta_gemm<double, false, true>(N, N, N, R.T, ld, Lf.T, ld, W1, ld, S.gemm);
  // 1/Db and Ds of both chains (vectors 5..7 of the workspace)
  double* ibR = wvec(C, s, 5);
  double* ibL = wvec(C, s, 6);
  for (int i = threadIdx.x; i < N; i += kThreads) {
    ibR[i] = 1.0 / (R.D[i] > 1.0 ? R.D[i] : 1.0);
    ibL[i] = 1.0 / (Lf.D[i] > 1.0 ? Lf.D[i] : 1.0);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < N * N; e += kThreads) {
    const int i = e / N, j = e - i * N;
    const double dR = R.D[i], dL = Lf.D[j];
    const double dsR = dR > 1.0 ? 1.0 : dR, dsL = dL > 1.0 ? 1.0 : dL;
    W0[(size_t)i * ld + j] = W0[(size_t)i * ld + j] * (ibR[i] * ibL[j]) + dsR * W1[(size_t)i * ld + j] * dsL;
  }
  __syncthreads();
  double ldm;
  int sm;
  int* piv = C.iwork[s] + ld;
  double* tmp = wmat(C, s, 9);
  if (lu_factor_blk(N, ld, W0, piv, tmp, ldm, sm, S)) return 1;
  int* rowof = C.iwork[s];
  lu_row_map(N, piv, rowof);
  for (int e = threadIdx.x; e < N * N; e += kThreads) {
    const int i = e / N, j = e - i * N;
    const int r = rowof[i];
    W1[(size_t)i * ld + j] = R.Q[(size_t)j * ld + r] * ibR[r];
  }
  __syncthreads();
  lu_solve_blk(N, ld, W0, W1, tmp, S);
  for (int e = threadIdx.x; e < N * N; e += kThreads) {
    const int i = e / N, j = e - i * N;
    W1[(size_t)i * ld + j] *= ibL[i];
  }
  __syncthreads();
  cta_gemm<double, false, false>(N, N, N, Lf.Q, ld, W1, ld, Gout, ld, S.gemm);
  double part = 0.0;
  for (int i = threadIdx.x; i < N; i += kThreads) {
    const double dR = R.D[i], dL = Lf.D[i];
    part += log(dR > 1.0 ? dR : 1.0) + log(dL > 1.0 ? dL : 1.0);
  }
  logdet = ldm + block_sum(part, S.red);
  sign = sm * R.detq * Lf.detq;
  return 0;
}

__device__ void copy_udv_to_slot(const ChainDev& C, int s, int j, int detq) {
  const int N = C.N, ld = C.ld;
  double* b = slot_base(C, s, j);
  cta_copy(N, ld, (const double*)wmat(C, s, 2), b);
  cta_copy(N, ld, (const double*)wmat(C, s, 5), b + (size_t)N * ld);
  const double* Dn = wvec(C, s, 0);
  for (int x = threadIdx.x; x < N; x += kThreads) b[(size_t)2 * N * ld + x] = Dn[x];
  if (threadIdx.x == 0) C.slot_detq[s][j] = detq;
  __syncthreads();
}

__device__ inline UDV work_udv(const ChainDev& C, int s, int detq) {
  UDV u;
  u.Q = wmat(C, s, 2);
  u.T = wmat(C, s, 5);
  u.D = wvec(C, s, 0);
  u.detq = detq;
  return u;
}

// Fill the storage with the left chain (Algorithm 1, the loop before the bins)
// and compute G(0) into W6.
__device__ int fill_left_chain(const ChainDev& C, int s, Smem& S, double& logdet, int& sign) {
  const int nst = C.L / C.nw;
  for (int j = nst - 1; j >= 0; --j) {
    const UDV src = (j + 1 == nst) ? ident_udv(C) : slot_udv(C, s, j + 1);
    const int dq = chain_step(C, s, j * C.nw, (j + 1) * C.nw, true, src, S);
    copy_udv_to_slot(C, s, j, dq);
  }
  return green_from_udv(C, s, ident_udv(C), slot_udv(C, s, 0), wmat(C, s, 6), logdet, sign, S);
}

// The float-pair stabilisation (defined with the mixed path below).
__device__ int chain_step_mixed(const ChainDev& C, int s, int t1, int t2, bool left, UDV src, Smem& S,
                                long long* det);
__device__ int green_from_udv_mixed(const ChainDev& C, int s, UDV R, UDV Lf, double* Gout, double& logdet,
                                    int& sign, Smem& S);

// Left chain and G(0) with the stabilisation arithmetic of the working
// precision: float pairs (FP64 scales) for the mixed paths, FP64 otherwise.
// Used when a chain starts or restarts from fields, so that the stored chain is
// the one the sweep itself would have left.
template <typename Real>
__device__ int fill_left_chain_working(const ChainDev& C, int s, Smem& S, double& logdet, int& sign) {
  if constexpr (std::is_same<Real, dd>::value) {
    const int nst = C.L / C.nw;
    for (int j = nst - 1; j >= 0; --j) {
      const UDV src = (j + 1 == nst) ? ident_udv(C) : slot_udv(C, s, j + 1);
      const int dq = chain_step_mixed(C, s, j * C.nw, (j + 1) * C.nw, true, src, S, nullptr);
      copy_udv_to_slot(C, s, j, dq);
    }
    return green_from_udv_mixed(C, s, ident_udv(C), slot_udv(C, s, 0), wmat(C, s, 6), logdet, sign, S);
  } else {
    return fill_left_chain(C, s, S, logdet, sign);
  }
}

// --------------------------------------------------------------------------
// Kernels templated on the working precision.
// --------------------------------------------------------------------------
// Fresh G(0) for every (chain, flavor): the left chain is (re)computed into the
// storage slots, G(0) lands in W6.  mode 0 (start from fields, in the working
// precision's stabilisation arithmetic): also write the working G, the
// fresh log|det| and the sign (initialisation); mode 1: copy G(0) of chain
// `out_chain` to `out` (FP64, [nfl][N][N]).
template <typename Real>
__global__ void __launch_bounds__(kThreads) fresh_green_kernel(ChainDev* chains, int n_chains, int mode,
                                                               double* out, int out_chain) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nfl = chains[0].nfl;
  const int c = blockIdx.x / nfl, s = blockIdx.x % nfl;
  if (c >= n_chains) return;
  if (mode == 1 && c != out_chain) return;
  ChainDev& C = chains[c];
  Smem S = carve_smem(smem_raw, C.ld, C.MV);
  // the working precision's tensor-core products need the CTA's tensor memory
  const bool umma = DQMC_WITH_UMMA && std::is_same<Real, dd>::value && mode == 0 && C.planes[s] != nullptr;
  S.um.err = &C.error;
  S.dd_tile = C.dd_tile;
  S.um.limit = C.wait_cycles > 0 ? C.wait_cycles : kUmmaWaitCycles;
  S.um.stall = C.test_stall;
  S.um.tmA = &C.tm_pl[s][0];
  S.um.tmB = &C.tm_pl[s][1];
  S.um.boff = (size_t)kUmmaDig * umma_pad(C.N, kUmmaM) * umma_pad(C.N, kUmmaK);
  S.um.where = C.wait_where[s];
  if (umma) umma_alloc(S.um);
  double logdet;
  int sign;
  const int bad = (mode == 0) ? fill_left_chain_working<Real>(C, s, S, logdet, sign)
                              : fill_left_chain(C, s, S, logdet, sign);
  if (umma) umma_free(S.um);
  if (bad) {
    if (threadIdx.x == 0) C.error = 1;
    return;
  }
  const double* Gf = wmat(C, s, 6);
  if (mode == 0) {
    Real* G = (Real*)C.G[s];
    for (int e = threadIdx.x; e < C.N * C.N; e += kThreads) {
      const int x = e / C.N, y = e - x * C.N;
      G[(size_t)x * C.ld + y] = from_d<Real>(Gf[(size_t)x * C.ld + y]);
    }
  } else {
    for (int e = threadIdx.x; e < C.N * C.N; e += kThreads) {
      const int x = e / C.N, y = e - x * C.N;
      out[(size_t)s * C.N * C.N + e] = Gf[(size_t)x * C.ld + y];
    }
  }
  if (threadIdx.x == 0) {
    C.logdet[s] = logdet;
    C.fresh_sign[s] = sign;
  }
}

// Hopping and potential wraps of one slice (defined with the sweep pieces below).
template <typename Real>
__device__ void v_wrap(const ChainDev& C, Real* G, const double* v, double a, Smem& S);
template <typename Real>
__device__ void t_wrap(const ChainDev& C, int s, Real* G, Real* Gt, bool up, Smem& S);

// G^s(tau) of one chain on its current fields as the upward pass of a sweep
// holds it when every proposal of the slices tau0+1..tau is rejected (Sec. 2.3,
// the wrapped Green function between stabilisations; Algorithm 1 wrapgrup):
// the stable G(tau0) at the last stabilisation point tau0 = n_wrap floor(tau /
// n_wrap), from the right chain B(tau0,0) built here and the stored left chain
// B(beta,tau0)^T, in the working precision's stabilisation arithmetic, then
// tau - tau0 wraps G <- E e^V G e^-V E^-1 in the working precision.  One CTA per
// flavor; the stored chain, the working G and the fields are only read.  Uses
// the work matrices W0..W8; out: [nfl][N][N] FP64.
template <typename Real>
__global__ void __launch_bounds__(kThreads) green_tau_kernel(ChainDev* chains, int chain, int tau, double* out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ChainDev& C = chains[chain];
  const int s = blockIdx.x;
  if (s >= C.nfl) return;
  Smem S = carve_smem(smem_raw, C.ld, C.MV);
  S.flavor = s;
  const int N = C.N, ld = C.ld, nw = C.nw, nst = C.L / nw;
  const int j0 = tau / nw;
  constexpr bool mixed = std::is_same<Real, dd>::value;
  const bool umma = DQMC_WITH_UMMA && mixed && C.planes[s] != nullptr;
  S.um.err = &C.error;
  S.dd_tile = C.dd_tile;
  S.um.limit = C.wait_cycles > 0 ? C.wait_cycles : kUmmaWaitCycles;
  S.um.stall = C.test_stall;
  S.um.tmA = &C.tm_pl[s][0];
  S.um.tmB = &C.tm_pl[s][1];
  S.um.boff = (size_t)kUmmaDig * umma_pad(C.N, kUmmaM) * umma_pad(C.N, kUmmaK);
  S.um.where = C.wait_where[s];
  if (umma) umma_alloc(S.um);
  int dq = 1;
  for (int j = 1; j <= j0; ++j) {
    const UDV src = (j == 1) ? ident_udv(C) : work_udv(C, s, dq);
    dq = mixed ? chain_step_mixed(C, s, (j - 1) * nw, j * nw, false, src, S, nullptr)
               : chain_step(C, s, (j - 1) * nw, j * nw, false, src, S);
  }
  const UDV R = (j0 == 0) ? ident_udv(C) : work_udv(C, s, dq);
  const UDV Lf = (j0 >= nst) ? ident_udv(C) : slot_udv(C, s, j0);
  double* Gf = wmat(C, s, 6);
  double logdet;
  int sg;
  const int bad = mixed ? green_from_udv_mixed(C, s, R, Lf, Gf, logdet, sg, S)
                        : green_from_udv(C, s, R, Lf, Gf, logdet, sg, S);
  if (bad) {
    if (umma) umma_free(S.um);
    if (threadIdx.x == 0) C.error = 1;
    return;
  }
  Real* G = reinterpret_cast<Real*>(wmat(C, s, 7));
  Real* Gt = reinterpret_cast<Real*>(wmat(C, s, 8));
  for (int e = threadIdx.x; e < N * N; e += kThreads) {
    const int x = e / N, y = e - x * N;
    G[(size_t)x * ld + y] = from_d<Real>(Gf[(size_t)x * ld + y]);
  }
  __syncthreads();
  for (int t = j0 * nw + 1; t <= tau; ++t) {
    slice_potential_global(C, s, t, S.v);
    v_wrap<Real>(C, G, S.v, +1.0, S);
    t_wrap<Real>(C, s, G, Gt, true, S);
  }
  if (umma) umma_free(S.um);
  for (int e = threadIdx.x; e < N * N; e += kThreads) {
    const int x = e / N, y = e - x * N;
    out[(size_t)s * N * N + e] = to_d(G[(size_t)x * ld + y]);
  }
}

template <typename Real>
__global__ void copy_green_kernel(ChainDev* chains, int chain, int flavor, double* out) {
  const ChainDev& C = chains[chain];
  const Real* G = (const Real*)C.G[flavor];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < C.N * C.N; e += gridDim.x * blockDim.x) {
    const int x = e / C.N, y = e - x * C.N;
    out[e] = to_d(G[(size_t)x * C.ld + y]);
  }
}

// ---- pieces of the sweep --------------------------------------------------

// G <- diag(ev) G diag(1/ev)  with ev = exp(a v)
template <typename Real>
__device__ void v_wrap(const ChainDev& C, Real* G, const double* v, double a, Smem& S) {
  const int N = C.N, ld = C.ld;
  Real* evr = reinterpret_cast<Real*>(S.ev);
  Real* evi = reinterpret_cast<Real*>(S.hv);
  for (int x = threadIdx.x; x < N; x += kThreads) {
    evr[x] = from_d<Real>(exp(a * v[x]));
    evi[x] = from_d<Real>(exp(-a * v[x]));
  }
  __syncthreads();
  for (int e = threadIdx.x; e < N * N; e += kThreads) {
    const int x = e / N, y = e - x * N;
    G[(size_t)x * ld + y] = rmul(rmul(G[(size_t)x * ld + y], evr[x]), evi[y]);
  }
  __syncthreads();
}

// Hopping wrap: up  G <- E G E^-1;  down  G <- E^-1 G E.
template <typename Real>
__device__ void t_wrap(const ChainDev& C, int s, Real* G, Real* Gt, bool up, Smem& S);

template <>
__device__ void t_wrap<double>(const ChainDev& C, int s, double* G, double* Gt, bool up, Smem& S) {
  const int N = C.N, ld = C.ld;
  const double* X = up ? C.E[s] : C.Einv[s];
  const double* Y = up ? C.Einv[s] : C.E[s];
  cta_gemm<double, false, false>(N, N, N, X, ld, G, ld, Gt, ld, S.gemm);
  cta_gemm<double, false, false>(N, N, N, Gt, ld, Y, ld, G, ld, S.gemm);
}
template <>
__device__ void t_wrap<float>(const ChainDev& C, int s, float* G, float* Gt, bool up, Smem& S) {
  const int N = C.N, ld = C.ld;
  const float* X = up ? C.E32[s] : C.Einv32[s];
  const float* Y = up ? C.Einv32[s] : C.E32[s];
  float* sm = reinterpret_cast<float*>(S.gemm);
  cta_gemm<float, false, false>(N, N, N, X, ld, G, ld, Gt, ld, sm);
  cta_gemm<float, false, false>(N, N, N, Gt, ld, Y, ld, G, ld, sm);
}

template <>
__device__ void t_wrap<dd>(const ChainDev& C, int s, dd* G, dd* Gt, bool up, Smem& S) {
  const int N = C.N, ld = C.ld;
  const dd* X = (const dd*)(up ? C.Edd[s] : C.Einvdd[s]);
  const dd* Y = (const dd*)(up ? C.Einvdd[s] : C.Edd[s]);
  gemm_dd<false, false, false>(C, s, S, N, N, N, X, ld, G, ld, Gt, ld, up ? kCpEA : kCpEiA, -1);
  gemm_dd<false, false, false>(C, s, S, N, N, N, Gt, ld, Y, ld, G, ld, -1, up ? kCpEiB : kCpEB);
}

// G <- G + sum_m a_m b_m^T  (flush of the delayed rank-k update), a register-
// blocked product G += A^T B with A, B stored as rows a_m, b_m.
template <typename Real>
__device__ void flush_delayed(const ChainDev& C, Real* G, const Real* A, const Real* B, int nacc, Smem& S);

template <>
__device__ void flush_delayed<double>(const ChainDev& C, double* G, const double* A, const double* B, int nacc,
                                      Smem& S) {
  const int N = C.N, ld = C.ld;
  const int r = gemm_pick_r(N);
  if (r == 3) cta_gemm_r<double, true, false, 3, true>(N, N, nacc, A, ld, B, ld, G, ld, S.gemm);
  else if (r == 5) cta_gemm_r<double, true, false, 5, true>(N, N, nacc, A, ld, B, ld, G, ld, S.gemm);
  else cta_gemm_r<double, true, false, 4, true>(N, N, nacc, A, ld, B, ld, G, ld, S.gemm);
}
template <>
__device__ void flush_delayed<float>(const ChainDev& C, float* G, const float* A, const float* B, int nacc,
                                     Smem& S) {
  const int N = C.N, ld = C.ld;
  float* sm = reinterpret_cast<float*>(S.gemm);
  const int r = gemm_pick_r(N);
  if (r == 3) cta_gemm_r<float, true, false, 3, true>(N, N, nacc, A, ld, B, ld, G, ld, sm);
  else if (r == 5) cta_gemm_r<float, true, false, 5, true>(N, N, nacc, A, ld, B, ld, G, ld, sm);
  else cta_gemm_r<float, true, false, 4, true>(N, N, nacc, A, ld, B, ld, G, ld, sm);
}
template <>
__device__ void flush_delayed<dd>(const ChainDev& C, dd* G, const dd* A, const dd* B, int nacc, Smem& S) {
  // a rank-k update (k <= 64): the float-pair SIMT tiles beat the split
  // tensor-core product, whose digit split and recombination cost O(N^2 k_dig)
  gemm_dd_tiles<true, false, true>(C.N, C.N, nacc, A, C.ld, B, C.ld, G, C.ld, reinterpret_cast<dd*>(S.gemm),
                                   S.dd_tile);
}

// Sequential single-field updates of one slice (Sec. 2.2.1) for this CTA's
// flavor.  The ratios of every remaining position are evaluated in parallel
// from the current diagonal of G; the first accepted position in visiting
// order is found by a block reduction, which is exactly the sequential
// Metropolis chain because rejected proposals leave G unchanged.  Accepted
// flips are applied as delayed rank-1 updates (flushed every k accepts):
//   a = -(delta/R_s) G_eff[:,i],  b = e_i - G_eff[i,:],  G_eff += a b^T.
template <typename Real>
__device__ void update_slice(ChainDev& C, int s, int tau, int dir, const SweepParams& P, Smem& S,
                             cg::cluster_group& cl, Real* G, Real* A, Real* B, int& sign, int& buf,
                             long long* det) {
  const int N = C.N, ld = C.ld, MV = C.MV, nfl = C.nfl, tid = threadIdx.x;
  long long t0 = clock64();
  const uint32_t key0 = (uint32_t)P.seed, key1 = (uint32_t)(P.seed >> 32) ^ C.chain_id;
  for (int q = tid; q < MV; q += kThreads) {
    const int k = dir ? MV - 1 - q : q;
    uint32_t ctr[4] = {(uint32_t)P.sweep, (uint32_t)(2 * tau + dir), (uint32_t)k, (uint32_t)(P.sweep >> 32)};
    philox4x32_10(ctr, key0, key1);
    const double u1 = uniform53(ctr[0], ctr[1]);
    S.u2[q] = uniform53(ctr[2], ctr[3]);
    const int f = S.fslice[k];
    const int fn = propose_field(C.ft, f, u1);
    const double dc = coupling(C.ft, C.cscale, fn) - coupling(C.ft, C.cscale, f);
    S.delta[q] = exp(C.vsign[s * MV + k] * dc) - 1.0;
    S.gam[q] = field_weight(C.ft, fn) / field_weight(C.ft, f);
    S.fnew[q] = (int8_t)fn;
    S.qsite[q] = C.site[k];
  }
  for (int x = tid; x < N; x += kThreads) {
    S.d[x] = to_d(G[(size_t)x * ld + x]);
    S.qinv[x] = -1;
  }
  // first accepted position of the current scan (two slots, alternating)
  int* first_slot = S.ired + 16;
  if (tid == 0) first_slot[0] = first_slot[1] = MV;
  __syncthreads();
  for (int q = tid; q < MV; q += kThreads) {
    S.qinv[S.qsite[q]] = q;
    S.Rs[buf * MV + q] = 1.0 + S.delta[q] * (1.0 - S.d[S.qsite[q]]);
  }
  __syncthreads();
  tick(det, 0, t0);
  int pos = 0, nacc = 0;
  int64_t n_acc_slice = 0;
  const int kdel = P.delay_k;
  // Barriers per acceptance: the cluster barrier (ratios of both flavors) and one
  // CTA barrier after the scan.  The thread that owns site x updates the
  // diagonal d_x and the next ratio of the vertex on x itself, so neither needs
  // a barrier of its own; the flush is preceded by one.
  while (true) {
    double* Rs = S.Rs + buf * MV;
    // the next position is accepted most of the time: start reading its column and
    // row of G now, so that the cluster barrier covers the memory latency
    const int ipre = (pos < MV) ? S.qsite[pos] : 0;
    Real gc_pre = from_d<Real>(0.0), gr_pre = from_d<Real>(0.0);
    if (tid < N) {
      gc_pre = G[(size_t)tid * ld + ipre];
      gr_pre = G[(size_t)ipre * ld + tid];
    }
    cl.sync();
    const double* Rr[kMaxFlavors];
    for (int r = 0; r < nfl; ++r) Rr[r] = (r == s) ? Rs : cl.map_shared_rank(Rs, r);
    for (int q = pos + tid; q < MV; q += kThreads) {
      double R = S.gam[q];
      for (int r = 0; r < nfl; ++r) R *= Rr[r][q];
      const double aR = fabs(R);
      if (S.u2[q] < (aR < 1.0 ? aR : 1.0)) {
        S.Rp[q] = R;
        atomicMin(first_slot + buf, q);
        break;
      }
    }
    __syncthreads();
    const int first = first_slot[buf];
    if (tid == 0) first_slot[buf ^ 1] = MV;
    tick(det, 1, t0);
    if (first >= MV) { buf ^= 1; break; }
    const double R = S.Rp[first];
    if (R < 0.0) sign = -sign;
    const int k = dir ? MV - 1 - first : first;
    const int i = S.qsite[first];
    const double fac = S.delta[first] / Rs[first];
    Real* a = A + (size_t)nacc * ld;
    Real* b = B + (size_t)nacc * ld;
    const Real mfac = from_d<Real>(-fac);
    const bool hit = (first == pos);
    double* Rs_next = S.Rs + (buf ^ 1) * MV;
    // element x of column i (a) and of row i (b) of G_eff
    for (int x = tid; x < N; x += kThreads) {
      Real cx, ry;
      if (hit && x == tid) {
        cx = gc_pre;
        ry = gr_pre;
      } else {
        cx = G[(size_t)x * ld + i];
        ry = G[(size_t)i * ld + x];
      }
      // two independent accumulation chains each (even and odd m)
      Real cx1 = from_d<Real>(0.0), ry1 = from_d<Real>(0.0);
      int m = 0;
      for (; m + 1 < nacc; m += 2) {
        cx = rfma(A[(size_t)m * ld + x], B[(size_t)m * ld + i], cx);
        ry = rfma(A[(size_t)m * ld + i], B[(size_t)m * ld + x], ry);
        cx1 = rfma(A[(size_t)(m + 1) * ld + x], B[(size_t)(m + 1) * ld + i], cx1);
        ry1 = rfma(A[(size_t)(m + 1) * ld + i], B[(size_t)(m + 1) * ld + x], ry1);
      }
      if (m < nacc) {
        cx = rfma(A[(size_t)m * ld + x], B[(size_t)m * ld + i], cx);
        ry = rfma(A[(size_t)m * ld + i], B[(size_t)m * ld + x], ry);
      }
      cx = radd(cx, cx1);
      ry = radd(ry, ry1);
      const Real ax = rmul(mfac, cx);
      const Real bx = rsub(from_d<Real>(x == i ? 1.0 : 0.0), ry);
      a[x] = ax;
      b[x] = bx;
      const double dx = S.d[x] + to_d(ax) * to_d(bx);
      S.d[x] = dx;
      const int qx = S.qinv[x];
      if (qx >= 0) Rs_next[qx] = 1.0 + S.delta[qx] * (1.0 - dx);
    }
    if (tid == 0) S.fslice[k] = S.fnew[first];
    ++nacc;
    ++n_acc_slice;
    tick(det, 2, t0);
    if (nacc == kdel) {
      __syncthreads();
      flush_delayed<Real>(C, G, A, B, nacc, S);
      nacc = 0;
      tick(det, 3, t0);
    }
    pos = first + 1;
    buf ^= 1;
  }
  if (nacc) flush_delayed<Real>(C, G, A, B, nacc, S);
  tick(det, 3, t0);
  if (s == 0 && tid == 0) {
    C.proposals += MV;
    C.accepted += n_acc_slice;
  }
}

// ---- float-pair Householder QR with FP64 column scales (mixed path) -------
// M = X diag(dsc) with X the float-pair product Bcal Q (entries O(1)) and dsc
// the FP64 scales D of the previous decomposition, which may exceed the float
// range.  Householder reflections act on rows and commute with the column
// scaling, so the pivoted QR of M is the QR of X with the pivot chosen by the
// scaled norm dsc_j ||X[k:, j]|| (Businger-Golub on M); R_M = R_X diag(dsc[perm]).
__device__ void householder_apply_dd(int N, int ld, dd* M, int k, int j0, dd bk, const dd* hv, dd* qred) {
  const int tid = threadIdx.x, lane = tid & 31, rg = tid >> 5;
  for (int c0 = j0; c0 < N; c0 += 128) {
    dd w[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    int i = k + rg;
    for (; i + 24 < N; i += 32) {
      dd x[4][4];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int j = c0 + lane + 32 * q;
          x[r][q] = (j < N) ? M[(size_t)(i + 8 * r) * ld + j] : dd{0.f, 0.f};
        }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const dd vi = hv[i + 8 * r];
#pragma unroll
        for (int q = 0; q < 4; ++q) w[q] = dd_fma(vi, x[r][q], w[q]);
      }
    }
    for (; i < N; i += 8) {
      const dd vi = hv[i];
      const dd* row = M + (size_t)i * ld;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int j = c0 + lane + 32 * q;
        if (j < N) w[q] = dd_fma(vi, row[j], w[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) qred[rg * 128 + lane + 32 * q] = w[q];
    __syncthreads();
    dd wt[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      dd t = {0.f, 0.f};
#pragma unroll
      for (int r = 0; r < 8; ++r) t = dd_add(t, qred[r * 128 + lane + 32 * q]);
      const dd bw = dd_mul(bk, t);
      wt[q] = {-bw.hi, -bw.lo};
    }
    i = k + rg;
    for (; i + 24 < N; i += 32) {
      dd x[4][4];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int j = c0 + lane + 32 * q;
          x[r][q] = (j < N) ? M[(size_t)(i + 8 * r) * ld + j] : dd{0.f, 0.f};
        }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const dd vi = hv[i + 8 * r];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int j = c0 + lane + 32 * q;
          if (j < N) M[(size_t)(i + 8 * r) * ld + j] = dd_fma(wt[q], vi, x[r][q]);
        }
      }
    }
    for (; i < N; i += 8) {
      const dd vi = hv[i];
      dd* row = M + (size_t)i * ld;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int j = c0 + lane + 32 * q;
        if (j < N) row[j] = dd_fma(wt[q], vi, row[j]);
      }
    }
    __syncthreads();
  }
}

__device__ int qr_pivoted_dd(int N, int ld, dd* X, double* dsc, double* beta, dd* vk0, double* cn_g, double* cn0_g,
                             int* perm_g, Smem& S) {
  // Per-column state in shared memory (the sweep's slice buffers, idle during
  // the stabilisation): norms cn / cn0, scales, pivot order, recompute list.
  // The reflector's scalars are formed by thread 0 and broadcast; the norms are
  // downdated with LAPACK's xGEQPF rule and those that cancel below its
  // threshold are recomputed in FP64 by one warp each.
  (void)cn_g;
  (void)cn0_g;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  dd* hv = reinterpret_cast<dd*>(S.hv);
  dd* qred = reinterpret_cast<dd*>(S.qred);
  double* cn = S.d;
  double* cn0 = S.xdiag;
  double* sd = S.ev;
  int* perm = S.qinv;
  int* flag = reinterpret_cast<int*>(S.spare);
  int* nflag = S.ired + 24;
  double* sc = S.xs + 4;
  for (int j = tid; j < N; j += kThreads) {
    double acc = 0.0;
    for (int i = 0; i < N; ++i) {
      const double x = to_d(X[(size_t)i * ld + j]);
      acc = fma(x, x, acc);
    }
    cn[j] = sqrt(acc);
    cn0[j] = cn[j];
    perm[j] = j;
    sd[j] = dsc[j];
  }
  __syncthreads();
  const double tol3z = sqrt(2.220446049250313e-16);
  int detq = 1;
  for (int k = 0; k < N; ++k) {
    double bv = -1.0;
    int bi = N;
    for (int j = k + tid; j < N; j += kThreads) {
      const double sn = sd[j] * cn[j];
      if (sn > bv) { bv = sn; bi = j; }
    }
    int p = block_argmax(bv, bi, S.red, S.ired);
    if (p >= N) p = k;
    if (p != k) {
      for (int i = tid; i < N; i += kThreads) {
        const dd t = X[(size_t)i * ld + k];
        X[(size_t)i * ld + k] = X[(size_t)i * ld + p];
        X[(size_t)i * ld + p] = t;
      }
      if (tid == 0) {
        const int tp = perm[k]; perm[k] = perm[p]; perm[p] = tp;
        double t = cn[k]; cn[k] = cn[p]; cn[p] = t;
        t = cn0[k]; cn0[k] = cn0[p]; cn0[p] = t;
        t = sd[k]; sd[k] = sd[p]; sd[p] = t;
      }
      __syncthreads();
    }
    double part = 0.0;
    for (int i = k + tid; i < N; i += kThreads) {
      const dd x = X[(size_t)i * ld + k];
      const double xd = to_d(x);
      part = fma(xd, xd, part);
      hv[i] = x;
    }
    const double xn2 = block_sum(part, S.red);
    if (tid == 0) {
      const double xnorm = sqrt(xn2);
      const dd x0 = hv[k];
      double bk = 0.0;
      if (xnorm > 0.0) {
        const double x0d = to_d(x0);
        const double alpha = (x0d >= 0.0) ? -xnorm : xnorm;
        const dd v0 = dd_add(x0, from_d<dd>(-alpha));
        const double v0d = to_d(v0);
        const double vtv = xn2 - x0d * x0d + v0d * v0d;
        bk = (vtv > 0.0) ? 2.0 / vtv : 0.0;
        hv[k] = v0;
        X[(size_t)k * ld + k] = from_d<dd>(alpha);
      }
      beta[k] = bk;
      vk0[k] = hv[k];
      sc[0] = bk;
      *nflag = 0;
    }
    __syncthreads();
    const double bk = sc[0];
    if (bk != 0.0) {
      detq = -detq;
      householder_apply_dd(N, ld, X, k, k + 1, from_d<dd>(bk), hv, qred);
    }
    for (int j = k + 1 + tid; j < N; j += kThreads) {
      if (cn[j] != 0.0) {
        double t = fabs(to_d(X[(size_t)k * ld + j])) / cn[j];
        t = fmax(0.0, (1.0 + t) * (1.0 - t));
        const double r = cn[j] / cn0[j];
        if (t * r * r <= tol3z) flag[atomicAdd(nflag, 1)] = j;
        else cn[j] *= sqrt(t);
      }
    }
    __syncthreads();
    const int nf = *nflag;
    if (nf) {
      for (int q = warp; q < nf; q += kThreads / 32) {
        const int j = flag[q];
        double acc = 0.0;
        for (int i = k + 1 + lane; i < N; i += 32) {
          const double x = to_d(X[(size_t)i * ld + j]);
          acc = fma(x, x, acc);
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
          cn[j] = sqrt(acc);
          cn0[j] = cn[j];
        }
      }
      __syncthreads();
    }
  }
  for (int j = tid; j < N; j += kThreads) {
    perm_g[j] = perm[j];
    dsc[j] = sd[j];
  }
  __syncthreads();
  return detq;
}

__device__ void form_q_dd(int N, int ld, const dd* X, const double* beta, const dd* vk0, dd* Q, Smem& S) {
  const int tid = threadIdx.x;
  dd* hv = reinterpret_cast<dd*>(S.hv);
  dd* qred = reinterpret_cast<dd*>(S.qred);
  for (int e = tid; e < N * N; e += kThreads) {
    const int x = e / N, y = e - x * N;
    Q[(size_t)x * ld + y] = {(x == y) ? 1.f : 0.f, 0.f};
  }
  __syncthreads();
  for (int k = N - 1; k >= 0; --k) {
    const double bk = beta[k];
    if (bk == 0.0) continue;
    for (int i = k + tid; i < N; i += kThreads) hv[i] = (i == k) ? vk0[k] : X[(size_t)i * ld + k];
    __syncthreads();
    householder_apply_dd(N, ld, Q, k, k, from_d<dd>(bk), hv, qred);
  }
}

// ---- stabilisation with float-float products (mixed path) ----------------
// Same steps as chain_step / green_from_udv; the dense products (the B chain,
// T = D^-1 R P^T T, Q_R^T Q_L, T_R T_L^T, Q_L Y) run as float-float GEMMs on the
// FP32 pipes, the pivoted QR, Q accumulation, LU and triangular solves stay
// FP64.  Storage matrices (Q, T) remain FP64.
__device__ inline void to_dd_mat(int N, int ld, const double* src, dd* dst) {
  for (int e = threadIdx.x; e < N * N; e += kThreads) {
    const int x = e / N, y = e - x * N;
    dst[(size_t)x * ld + y] = from_d<dd>(src[(size_t)x * ld + y]);
  }
  __syncthreads();
}

// dd -> double in place (same 8-byte slot)
__device__ inline void dd_to_d_inplace(int N, int ld, void* buf) {
  dd* a = reinterpret_cast<dd*>(buf);
  double* b = reinterpret_cast<double*>(buf);
  for (int e = threadIdx.x; e < N * N; e += kThreads) {
    const int x = e / N, y = e - x * N;
    const dd v = a[(size_t)x * ld + y];
    b[(size_t)x * ld + y] = to_d(v);
  }
  __syncthreads();
}

__device__ int chain_step_mixed(const ChainDev& C, int s, int t1, int t2, bool left, UDV src, Smem& S,
                      long long* det = nullptr) {
  long long t0 = clock64();
  const int N = C.N, ld = C.ld;
  dd* X = reinterpret_cast<dd*>(wmat(C, s, 0));
  dd* Y = reinterpret_cast<dd*>(wmat(C, s, 1));
  dd* evr = reinterpret_cast<dd*>(S.ev);
  to_dd_mat(N, ld, src.Q, X);
  const dd* E = (const dd*)C.Edd[s];
  if (!left) {
    for (int t = t1 + 1; t <= t2; ++t) {
      slice_potential_global(C, s, t, S.v);
      for (int x = threadIdx.x; x < N; x += kThreads) evr[x] = from_d<dd>(exp(S.v[x]));
      __syncthreads();
      for (int e = threadIdx.x; e < N * N; e += kThreads) {
        const int x = e / N, y = e - x * N;
        X[(size_t)x * ld + y] = dd_mul(X[(size_t)x * ld + y], evr[x]);
      }
      __syncthreads();
      gemm_dd<false, false, false>(C, s, S, N, N, N, E, ld, X, ld, Y, ld, kCpEA, -1);
      dd* t_ = X; X = Y; Y = t_;
    }
  } else {
    for (int t = t2; t >= t1 + 1; --t) {
      gemm_dd<true, false, false>(C, s, S, N, N, N, E, ld, X, ld, Y, ld, kCpEtA, -1);
      slice_potential_global(C, s, t, S.v);
      for (int x = threadIdx.x; x < N; x += kThreads) evr[x] = from_d<dd>(exp(S.v[x]));
      __syncthreads();
      for (int e = threadIdx.x; e < N * N; e += kThreads) {
        const int x = e / N, y = e - x * N;
        Y[(size_t)x * ld + y] = dd_mul(Y[(size_t)x * ld + y], evr[x]);
      }
      __syncthreads();
      dd* t_ = X; X = Y; Y = t_;
    }
  }
  tick(det, 4, t0);
  double* Dn = wvec(C, s, 0);
  double* beta = wvec(C, s, 1);
  dd* vk0 = reinterpret_cast<dd*>(wvec(C, s, 2));
  double* dsc = wvec(C, s, 5);
  double* invr = wvec(C, s, 6);
  int* perm = C.iwork[s];
  for (int j = threadIdx.x; j < N; j += kThreads) dsc[j] = src.D[j];
  __syncthreads();
  const int detq = qr_pivoted_dd(N, ld, X, dsc, beta, vk0, wvec(C, s, 3), wvec(C, s, 4), perm, S);
  dd* Qd = reinterpret_cast<dd*>(wmat(C, s, 2));
  form_q_dd(N, ld, X, beta, vk0, Qd, S);
  dd_to_d_inplace(N, ld, Qd);
  tick(det, 5, t0);
  dd* PT = reinterpret_cast<dd*>(wmat(C, s, 3));
  dd* Rt = reinterpret_cast<dd*>(wmat(C, s, 4));
  // D = |diag R_M| = |R_X,kk| dsc_k;  R~_ij = R_X,ij dsc_j / (|R_X,ii| dsc_i), |R~_ij| <= 1
  for (int x = threadIdx.x; x < N; x += kThreads) {
    const double rkk = fabs(to_d(X[(size_t)x * ld + x]));
    Dn[x] = rkk * dsc[x];
    invr[x] = (rkk > 0.0 && dsc[x] > 0.0) ? 1.0 / (rkk * dsc[x]) : 0.0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < N * N; e += kThreads) {
    const int x = e / N, y = e - x * N;
    PT[(size_t)x * ld + y] = from_d<dd>(src.T[(size_t)perm[x] * ld + y]);
    dd r = {0.f, 0.f};
    if (y >= x) r = dd_mul(X[(size_t)x * ld + y], from_d<dd>(invr[x] * dsc[y]));
    Rt[(size_t)x * ld + y] = r;
  }
  __syncthreads();
  dd* Tn = reinterpret_cast<dd*>(wmat(C, s, 5));
  gemm_dd<false, false, false>(C, s, S, N, N, N, Rt, ld, PT, ld, Tn, ld);
  dd_to_d_inplace(N, ld, Tn);
  tick(det, 6, t0);
  return detq;
}

__device__ int green_from_udv_mixed(const ChainDev& C, int s, UDV R, UDV Lf, double* Gout, double& logdet,
                                    int& sign, Smem& S) {
  const int N = C.N, ld = C.ld;
  dd* W0d = reinterpret_cast<dd*>(wmat(C, s, 0));
  dd* W1d = reinterpret_cast<dd*>(wmat(C, s, 1));
  dd* QRd = reinterpret_cast<dd*>(wmat(C, s, 3));
  dd* QLd = reinterpret_cast<dd*>(wmat(C, s, 4));
  dd* TRd = reinterpret_cast<dd*>(wmat(C, s, 7));
  dd* TLd = reinterpret_cast<dd*>(wmat(C, s, 8));
  to_dd_mat(N, ld, R.Q, QRd);
  to_dd_mat(N, ld, Lf.Q, QLd);
  to_dd_mat(N, ld, R.T, TRd);
  to_dd_mat(N, ld, Lf.T, TLd);
  gemm_dd<true, false, false>(C, s, S, N, N, N, QRd, ld, QLd, ld, W0d, ld);
  gemm_dd<false, true, false>(C, s, S, N, N, N, TRd, ld, TLd, ld, W1d, ld);
  double* ibR = wvec(C, s, 5);
  double* ibL = wvec(C, s, 6);
  for (int i = threadIdx.x; i < N; i += kThreads) {
    ibR[i] = 1.0 / (R.D[i] > 1.0 ? R.D[i] : 1.0);
    ibL[i] = 1.0 / (Lf.D[i] > 1.0 ? Lf.D[i] : 1.0);
  }
  __syncthreads();
  // Mid (float pairs, scale factors applied in FP64) in W0; right-hand side in W1
  for (int e = threadIdx.x; e < N * N; e += kThreads) {
    const int i = e / N, j = e - i * N;
    const double dR = R.D[i], dL = Lf.D[j];
    const double dsR = dR > 1.0 ? 1.0 : dR, dsL = dL > 1.0 ? 1.0 : dL;
    const double qq = to_d(W0d[(size_t)i * ld + j]);
    const double tt = to_d(W1d[(size_t)i * ld + j]);
    W0d[(size_t)i * ld + j] = from_d<dd>(qq * (ibR[i] * ibL[j]) + dsR * tt * dsL);
  }
  __syncthreads();
  double ldm;
  int smi;
  int* piv = C.iwork[s] + ld;
  dd* tmpd = reinterpret_cast<dd*>(wmat(C, s, 9));
  if (lu_factor_blk(N, ld, W0d, piv, tmpd, ldm, smi, S)) return 1;
  // right-hand side Db_R^-1 Q_R^T with the LU row interchanges applied
  int* rowof = C.iwork[s];
  lu_row_map(N, piv, rowof);
  for (int e = threadIdx.x; e < N * N; e += kThreads) {
    const int i = e / N, j = e - i * N;
    const int r = rowof[i];
    W1d[(size_t)i * ld + j] = from_d<dd>(R.Q[(size_t)j * ld + r] * ibR[r]);
  }
  __syncthreads();
  lu_solve_blk(N, ld, W0d, W1d, tmpd, S);
  dd* Yd = reinterpret_cast<dd*>(wmat(C, s, 9));
  for (int e = threadIdx.x; e < N * N; e += kThreads) {
    const int i = e / N, j = e - i * N;
    Yd[(size_t)i * ld + j] = from_d<dd>(to_d(W1d[(size_t)i * ld + j]) * ibL[i]);
  }
  __syncthreads();
  gemm_dd<false, false, false>(C, s, S, N, N, N, QLd, ld, Yd, ld, reinterpret_cast<dd*>(Gout), ld);
  dd_to_d_inplace(N, ld, Gout);
  double part = 0.0;
  for (int i = threadIdx.x; i < N; i += kThreads) {
    const double dR = R.D[i], dL = Lf.D[i];
    part += log(dR > 1.0 ? dR : 1.0) + log(dL > 1.0 ? dL : 1.0);
  }
  logdet = ldm + block_sum(part, S.red);
  sign = smi * R.detq * Lf.detq;
  return 0;
}

// Stabilisation event of this CTA's flavor at slice tau: new chain, fresh G,
// precision monitor, working G replaced, storage slot j written.
template <typename Real>
__device__ void stabilise(ChainDev& C, int s, int j, bool up, Real* G, Smem& S, double& ev_max,
                          double& ev_sum, int& fresh_sign, long long* det) {
  long long t0 = clock64();
  const int N = C.N, ld = C.ld, nst = C.L / C.nw, nw = C.nw;
  int dq;
  UDV R, Lf;
  constexpr bool mixed = std::is_same<Real, dd>::value;
  if (up) {
    const UDV src = (j == 1) ? ident_udv(C) : slot_udv(C, s, j - 1);
    dq = mixed ? chain_step_mixed(C, s, (j - 1) * nw, j * nw, false, src, S, det)
               : chain_step(C, s, (j - 1) * nw, j * nw, false, src, S, det);
    R = work_udv(C, s, dq);
    Lf = (j == nst) ? ident_udv(C) : slot_udv(C, s, j);
  } else {
    const UDV src = (j + 1 == nst) ? ident_udv(C) : slot_udv(C, s, j + 1);
    dq = mixed ? chain_step_mixed(C, s, j * nw, (j + 1) * nw, true, src, S, det)
               : chain_step(C, s, j * nw, (j + 1) * nw, true, src, S, det);
    Lf = work_udv(C, s, dq);
    R = (j == 0) ? ident_udv(C) : slot_udv(C, s, j);
  }
  t0 = clock64();
  double* Gf = wmat(C, s, 6);
  double logdet;
  int sg;
  const int bad = mixed ? green_from_udv_mixed(C, s, R, Lf, Gf, logdet, sg, S)
                        : green_from_udv(C, s, R, Lf, Gf, logdet, sg, S);
  if (bad) {
    if (threadIdx.x == 0) C.error = 1;
    sg = 1;
  }
  tick(det, 7, t0);
  double mx = 0.0, sm = 0.0;
  for (int e = threadIdx.x; e < N * N; e += kThreads) {
    const int x = e / N, y = e - x * N;
    const double gf = Gf[(size_t)x * ld + y];
    const double dg = fabs(gf - to_d(G[(size_t)x * ld + y]));
    mx = fmax(mx, dg);
    sm += dg;
    G[(size_t)x * ld + y] = from_d<Real>(gf);
  }
  ev_max = block_max(mx, S.red);
  ev_sum = block_sum(sm, S.red);
  fresh_sign = sg;
  if (threadIdx.x == 0) {
    C.logdet[s] = logdet;
    C.fresh_sign[s] = sg;
  }
  copy_udv_to_slot(C, s, j, dq);
}

// Energy estimator at the current G (Sec. 6 observables, U n_up n_dn form).
template <typename Real>
__device__ void measure(ChainDev& C, int s, const Real* G, Smem& S, cg::cluster_group& cl, int sign) {
  const int N = C.N, ld = C.ld;
  const double* K = C.K[s];
  double kin = 0.0, part = 0.0;
  for (int e = threadIdx.x; e < N * N; e += kThreads) {
    const int x = e / N, y = e - x * N;
    kin += K[(size_t)x * ld + y] * ((x == y ? 1.0 : 0.0) - to_d(G[(size_t)y * ld + x]));
  }
  for (int x = threadIdx.x; x < N; x += kThreads) {
    const double gxx = to_d(G[(size_t)x * ld + x]);
    part += 1.0 - gxx;
    S.xdiag[x] = gxx;
  }
  kin = block_sum(kin, S.red);
  part = block_sum(part, S.red);
  if (threadIdx.x == 0) { S.xs[0] = kin; S.xs[1] = part; }
  cl.sync();
  if (s == 0) {
    double pot = 0.0;
    if (C.nfl == 2) {
      const double* pd = cl.map_shared_rank(S.xdiag, 1);
      for (int x = threadIdx.x; x < N; x += kThreads) pot += C.U * (1.0 - S.xdiag[x]) * (1.0 - pd[x]);
    }
    pot = block_sum(pot, S.red);
    double kin_t = S.xs[0], part_t = S.xs[1];
    if (C.nfl == 2) {
      const double* px = cl.map_shared_rank(S.xs, 1);
      kin_t += px[0];
      part_t += px[1];
    }
    if (threadIdx.x == 0) {
      const double sg = (double)sign;
      C.meas[0] += sg * kin_t;
      C.meas[1] += sg * pot;
      C.meas[2] += sg * part_t;
      C.meas[3] += sg * (kin_t + pot);
      C.meas_sign += sg;
      C.n_meas += 1;
    }
  }
  cl.sync();
}

// Exchange this flavor's fresh sign and precision figures; returns the product
// of the fresh signs.  Rank 0 books the event.
__device__ int close_event(ChainDev& C, int s, Smem& S, cg::cluster_group& cl, double ev_max, double ev_sum,
                           int fresh_sign, int sign) {
  if (threadIdx.x == 0) S.xs[2] = (double)fresh_sign;
  cl.sync();
  int prod = 1;
  for (int r = 0; r < C.nfl; ++r) {
    const double* px = (r == s) ? S.xs : cl.map_shared_rank(S.xs, r);
    prod *= (px[2] < 0.0) ? -1 : 1;
  }
  if (threadIdx.x == 0) {
    C.prec_sum[s] += ev_sum / ((double)C.N * C.N * C.nfl);
    C.prec_max[s] = fmax(C.prec_max[s], ev_max);
    if (s == 0) {
      C.phase_max = fmax(C.phase_max, fabs((double)prod - (double)sign));
      C.prec_events += 1;
    }
  }
  cl.sync();
  return prod;
}

// One sweep of every chain (Algorithm 1, upward then downward).
template <typename Real>
__global__ void __launch_bounds__(kThreads, 2) sweep_kernel(ChainDev* chains, SweepParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cg::cluster_group cl = cg::this_cluster();
  const int nfl = (int)cl.num_blocks();
  const int s = (int)cl.block_rank();
  const int c = P.order[blockIdx.x / nfl];
  ChainDev& C = chains[c];
  Smem S = carve_smem(smem_raw, C.ld, C.MV);
  S.flavor = s;
  // the split tensor-core products (float-pair path with digit planes) need the
  // CTA's tensor memory for the whole sweep
  const bool umma = DQMC_WITH_UMMA && std::is_same<Real, dd>::value && C.planes[s] != nullptr;
  S.um.err = &C.error;
  S.dd_tile = C.dd_tile;
  S.um.limit = C.wait_cycles > 0 ? C.wait_cycles : kUmmaWaitCycles;
  S.um.stall = C.test_stall;
  S.um.tmA = &C.tm_pl[s][0];
  S.um.tmB = &C.tm_pl[s][1];
  S.um.boff = (size_t)kUmmaDig * umma_pad(C.N, kUmmaM) * umma_pad(C.N, kUmmaK);
  S.um.where = C.wait_where[s];
  if (umma) umma_alloc(S.um);
  Real* G = (Real*)C.G[s];
  Real* Gt = (Real*)C.Gtmp[s];
  Real* A = P.ab_smem ? reinterpret_cast<Real*>(S.ab) : (Real*)C.dA[s];
  Real* B = P.ab_smem ? A + (size_t)P.delay_k * C.ld : (Real*)C.dB[s];
  const int L = C.L, nw = C.nw, MV = C.MV;
  int sign = C.sign;
  int buf = 0;
  // thread 0's phase counters: cyc[0..3] per phase, det[0..7] per sub-phase
  long long* cyc = reinterpret_cast<long long*>(smem_raw);
  long long* det = cyc + 4;
  if (threadIdx.x == 0)
    for (int q = 0; q < 12; ++q) cyc[q] = 0;
  long long t0 = clock64();
  auto lap = [&](int phase) {
    const long long t1 = clock64();
    if (threadIdx.x == 0) cyc[phase] += t1 - t0;
    t0 = t1;
  };
  for (int tau = 1; tau <= L; ++tau) {
    for (int k = threadIdx.x; k < MV; k += kThreads) S.fslice[k] = C.fields[(size_t)(tau - 1) * MV + k];
    __syncthreads();
    slice_potential_smem(C, s, S.fslice, S.v);
    v_wrap<Real>(C, G, S.v, +1.0, S);
    lap(1);
    update_slice<Real>(C, s, tau, 0, P, S, cl, G, A, B, sign, buf, det);
    if (s == 0)
      for (int k = threadIdx.x; k < MV; k += kThreads) C.fields[(size_t)(tau - 1) * MV + k] = S.fslice[k];
    lap(0);
    t_wrap<Real>(C, s, G, Gt, true, S);
    lap(1);
    if (tau % nw == 0) {
      cl.sync();
      double mx, sm;
      int fs;
      stabilise<Real>(C, s, tau / nw, true, G, S, mx, sm, fs, det);
      sign = close_event(C, s, S, cl, mx, sm, fs, sign);
      lap(2);
    }
    if (P.measure && tau >= P.meas_first && tau <= P.meas_last) {
      measure<Real>(C, s, G, S, cl, sign);
      lap(3);
    }
  }
  for (int tau = L; tau >= 1; --tau) {
    for (int k = threadIdx.x; k < MV; k += kThreads) S.fslice[k] = C.fields[(size_t)(tau - 1) * MV + k];
    __syncthreads();
    t_wrap<Real>(C, s, G, Gt, false, S);
    lap(1);
    update_slice<Real>(C, s, tau, 1, P, S, cl, G, A, B, sign, buf, det);
    if (s == 0)
      for (int k = threadIdx.x; k < MV; k += kThreads) C.fields[(size_t)(tau - 1) * MV + k] = S.fslice[k];
    lap(0);
    slice_potential_smem(C, s, S.fslice, S.v);
    v_wrap<Real>(C, G, S.v, -1.0, S);
    lap(1);
    const int t0s = tau - 1;
    if (t0s % nw == 0) {
      cl.sync();
      double mx, sm;
      int fs;
      stabilise<Real>(C, s, t0s / nw, false, G, S, mx, sm, fs, det);
      sign = close_event(C, s, S, cl, mx, sm, fs, sign);
      lap(2);
    }
    if (P.measure && t0s >= P.meas_first && t0s <= P.meas_last) {
      measure<Real>(C, s, G, S, cl, sign);
      lap(3);
    }
  }
  cl.sync();
  if (umma) umma_free(S.um);
  if (threadIdx.x == 0) {
    for (int q = 0; q < 4; ++q) C.cyc[s][q] += cyc[q];
    for (int q = 0; q < 8; ++q) C.cycd[s][q] += det[q];
    if (s == 0) {
      C.sign = sign;
      C.sweep_sign_sum += (double)sign;
    }
  }
}

// --------------------------------------------------------------------------
// Launch helpers (instantiated once per precision unit).
// --------------------------------------------------------------------------
static inline cudaError_t set_smem(const void* fn, size_t bytes) {
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename Real>
static cudaError_t launch_fresh_green_t(ChainDev* chains, int n_chains, int nfl, size_t smem, int mode,
                                        double* out, int out_chain, cudaStream_t st) {
  cudaError_t e = set_smem((const void*)fresh_green_kernel<Real>, smem);
  if (e != cudaSuccess) return e;
  fresh_green_kernel<Real><<<n_chains * nfl, kThreads, smem, st>>>(chains, n_chains, mode, out, out_chain);
  return cudaGetLastError();
}

template <typename Real>
static cudaError_t launch_green_tau_t(ChainDev* chains, int chain, int nfl, size_t smem, int tau, double* out,
                                      cudaStream_t st) {
  cudaError_t e = set_smem((const void*)green_tau_kernel<Real>, smem);
  if (e != cudaSuccess) return e;
  green_tau_kernel<Real><<<nfl, kThreads, smem, st>>>(chains, chain, tau, out);
  return cudaGetLastError();
}

template <typename Real>
static cudaError_t launch_sweep_t(ChainDev* chains, const SweepParams& p, int nfl, size_t smem,
                                  cudaStream_t st) {
  cudaError_t e = set_smem((const void*)sweep_kernel<Real>, smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(p.n_chains * nfl, 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = nfl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, sweep_kernel<Real>, chains, p);
}

// Time-displaced Green functions from the two chains, sharing the middle
// matrix of the stable G (Sec. 2.1 observables, two times):
//   G(tau,0) = Q_L Db_L^-1 Mid^-1 Ds_R T_R,
//   G(0,tau) = -T_L^T Ds_L Mid^-1 Db_R^-1 Q_R^T.
// Uses W0, W1, W7, W8.  Returns nonzero if Mid is singular.
__device__ int displaced_from_udv(const ChainDev& C, int s, UDV R, UDV Lf, double* Gt0, double* G0t, Smem& S) {
  const int N = C.N, ld = C.ld;
  double* W0 = wmat(C, s, 0);
  double* W1 = wmat(C, s, 1);
  double* W7 = wmat(C, s, 7);
  double* W8 = wmat(C, s, 8);
  cta_gemm<double, true, false>(N, N, N, R.Q, ld, Lf.Q, ld, W0, ld, S.gemm);
  cta_gemm<double, false, true>(N, N, N, R.T, ld, Lf.T, ld, W1, ld, S.gemm);
  for (int e = threadIdx.x; e < N * N; e += kThreads) {
    const int i = e / N, j = e - i * N;
    const double dR = R.D[i], dL = Lf.D[j];
    const double dbR = dR > 1.0 ? dR : 1.0, dsR = dR > 1.0 ? 1.0 : dR;
    const double dbL = dL > 1.0 ? dL : 1.0, dsL = dL > 1.0 ? 1.0 : dL;
    W0[(size_t)i * ld + j] = W0[(size_t)i * ld + j] / (dbR * dbL) + dsR * W1[(size_t)i * ld + j] * dsL;
  }
  __syncthreads();
  double ldm;
  int smi;
  int* piv = C.iwork[s] + ld;
  double* tmp = wmat(C, s, 9);
  if (lu_factor_blk(N, ld, W0, piv, tmp, ldm, smi, S)) return 1;
  int* rowof = C.iwork[s];
  lu_row_map(N, piv, rowof);
  for (int e = threadIdx.x; e < N * N; e += kThreads) {
    const int i = e / N, j = e - i * N;
    W1[(size_t)i * ld + j] = (rowof[i] == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  lu_solve_blk(N, ld, W0, W1, tmp, S);  // W1 = Mid^-1
  for (int e = threadIdx.x; e < N * N; e += kThreads) {
    const int i = e / N, j = e - i * N;
    const double m = W1[(size_t)i * ld + j];
    const double dLi = Lf.D[i], dRj = R.D[j];
    W7[(size_t)i * ld + j] = m / (dLi > 1.0 ? dLi : 1.0) * (dRj > 1.0 ? 1.0 : dRj);
    W8[(size_t)i * ld + j] = (dLi > 1.0 ? 1.0 : dLi) * m / (dRj > 1.0 ? dRj : 1.0);
  }
  __syncthreads();
  cta_gemm<double, false, false>(N, N, N, Lf.Q, ld, W7, ld, W0, ld, S.gemm);
  cta_gemm<double, false, false>(N, N, N, W0, ld, R.T, ld, Gt0, ld, S.gemm);
  cta_gemm<double, true, false>(N, N, N, Lf.T, ld, W8, ld, W0, ld, S.gemm);
  cta_gemm<double, false, true>(N, N, N, W0, ld, R.Q, ld, G0t, ld, S.gemm);
  for (int e = threadIdx.x; e < N * N; e += kThreads) {
    const int i = e / N, j = e - i * N;
    G0t[(size_t)i * ld + j] = -G0t[(size_t)i * ld + j];
  }
  __syncthreads();
  return 0;
}

}  // namespace

size_t get_smem_bytes();  // dynamic shared memory of the fresh-G / adjoint / measurement kernels

// One pair per precision unit: 0 = FP64, 1 = FP32, 2/3 = float-pair (mixed).
cudaError_t launch_sweep_fp64(ChainDev* chains, const SweepParams& p, int nfl, size_t smem, cudaStream_t st);
cudaError_t launch_sweep_fp32(ChainDev* chains, const SweepParams& p, int nfl, size_t smem, cudaStream_t st);
cudaError_t launch_sweep_mixed(ChainDev* chains, const SweepParams& p, int nfl, size_t smem, cudaStream_t st);
cudaError_t launch_fresh_green_fp64(ChainDev* chains, int n_chains, int nfl, size_t smem, int mode, double* out,
                                    int out_chain, cudaStream_t st);
cudaError_t launch_fresh_green_fp32(ChainDev* chains, int n_chains, int nfl, size_t smem, int mode, double* out,
                                    int out_chain, cudaStream_t st);
cudaError_t launch_fresh_green_mixed(ChainDev* chains, int n_chains, int nfl, size_t smem, int mode, double* out,
                                     int out_chain, cudaStream_t st);
cudaError_t launch_green_tau_fp64(ChainDev* chains, int chain, int nfl, size_t smem, int tau, double* out,
                                  cudaStream_t st);
cudaError_t launch_green_tau_fp32(ChainDev* chains, int chain, int nfl, size_t smem, int tau, double* out,
                                  cudaStream_t st);
cudaError_t launch_green_tau_mixed(ChainDev* chains, int chain, int nfl, size_t smem, int tau, double* out,
                                   cudaStream_t st);
cudaError_t launch_sweep_mixed_tc(ChainDev* chains, const SweepParams& p, int nfl, size_t smem, cudaStream_t st);
cudaError_t launch_fresh_green_mixed_tc(ChainDev* chains, int n_chains, int nfl, size_t smem, int mode, double* out,
                                        int out_chain, cudaStream_t st);
cudaError_t launch_green_tau_mixed_tc(ChainDev* chains, int chain, int nfl, size_t smem, int tau, double* out,
                                      cudaStream_t st);

}  // namespace dqmc
