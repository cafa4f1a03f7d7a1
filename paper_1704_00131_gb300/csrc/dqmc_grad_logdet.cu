// Adjoint of log|det(1 + B(beta,0))| on fixed fields: hopping through the
// Frechet derivative of exp(-dtau K), coupling through dc/dU.
#include "dqmc_device.cuh"

namespace dqmc {

// d log|det(1 + B^s(beta,0))| on fixed fields: walk tau upwards with wraps
// and fresh recomputes at the stabilisation points, accumulating
//   S = sum_tau (1 - Gt_tau),  Gt_tau = e^{V_tau} G(tau-1) e^{-V_tau},
//   gU = sum_tau sum_k (1 - Gt_tau)_ii sigma_k dc(f_k,tau)/dU,
// then grad_K = V [F o (V^T (S E^-1)^T V)] V^T with the divided differences
// F of exp(-dtau x) over the eigenvalues of K (Frechet derivative).
__global__ void __launch_bounds__(kThreads) logdet_grad_kernel(ChainDev* chains, int n_cfg, const double* V,
                                                               const double* w, double* gK, double* gU) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nfl = chains[0].nfl;
  const int c = blockIdx.x / nfl, s = blockIdx.x % nfl;
  if (c >= n_cfg) return;
  ChainDev& C = chains[c];
  Smem S = carve_smem(smem_raw, C.ld, C.MV);
  const int N = C.N, ld = C.ld, L = C.L, nw = C.nw, nst = L / nw;
  double logdet;
  int sign;
  if (fill_left_chain(C, s, S, logdet, sign)) {
    if (threadIdx.x == 0) C.error = 1;
    return;
  }
  if (threadIdx.x == 0) { C.logdet[s] = logdet; C.fresh_sign[s] = sign; }
  double* Gc = wmat(C, s, 7);
  double* Sacc = wmat(C, s, 8);
  double* Wt = wmat(C, s, 9);
  cta_copy(N, ld, (const double*)wmat(C, s, 6), Gc);
  for (int e = threadIdx.x; e < N * N; e += kThreads) {
    const int x = e / N, y = e - x * N;
    Sacc[(size_t)x * ld + y] = 0.0;
  }
  __syncthreads();
  double gu = 0.0;
  for (int tau = 1; tau <= L; ++tau) {
    slice_potential_global(C, s, tau, S.v);
    for (int x = threadIdx.x; x < N; x += kThreads) S.ev[x] = exp(S.v[x]);
    __syncthreads();
    for (int e = threadIdx.x; e < N * N; e += kThreads) {
      const int x = e / N, y = e - x * N;
      const double gt = Gc[(size_t)x * ld + y] * (S.ev[x] / S.ev[y]);
      Gc[(size_t)x * ld + y] = gt;
      Sacc[(size_t)x * ld + y] += (x == y ? 1.0 : 0.0) - gt;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < C.MV; k += kThreads) {
      const int i = C.site[k];
      gu += (1.0 - Gc[(size_t)i * ld + i]) * C.vsign[s * C.MV + k] *
            coupling_dU(C.ft, C.dtau, C.U, C.cscale, C.fields[(size_t)(tau - 1) * C.MV + k]);
    }
    cta_gemm<double, false, false>(N, N, N, C.E[s], ld, Gc, ld, Wt, ld, S.gemm);
    cta_gemm<double, false, false>(N, N, N, Wt, ld, C.Einv[s], ld, Gc, ld, S.gemm);
    if (tau % nw == 0 && tau < L) {
      const int j = tau / nw;
      const UDV src = (j == 1) ? ident_udv(C) : slot_udv(C, s, j - 1);
      const int dq = chain_step(C, s, (j - 1) * nw, j * nw, false, src, S);
      const UDV Lf = (j == nst) ? ident_udv(C) : slot_udv(C, s, j);
      double ldt;
      int sgt;
      if (green_from_udv(C, s, work_udv(C, s, dq), Lf, wmat(C, s, 6), ldt, sgt, S)) {
        if (threadIdx.x == 0) C.error = 1;
        return;
      }
      cta_copy(N, ld, (const double*)wmat(C, s, 6), Gc);
      copy_udv_to_slot(C, s, j, dq);
    }
  }
  gu = block_sum(gu, S.red);
  if (threadIdx.x == 0) gU[(size_t)c * nfl + s] = gu;
  // A = S E^-1 -> W0;  W1 = A^T V;  W2 = V^T W1;  F o W2;  W1 = V W2;  W3 = W1 V^T
  double* W0 = wmat(C, s, 0);
  double* W1 = wmat(C, s, 1);
  double* W2 = wmat(C, s, 2);
  double* W3 = wmat(C, s, 3);
  const double* Vs = V + (size_t)s * N * N;
  const double* ws = w + (size_t)s * N;
  cta_gemm<double, false, false>(N, N, N, Sacc, ld, C.Einv[s], ld, W0, ld, S.gemm);
  // V is dense [N][N] (ld = N); use a copy with the chain's ld
  for (int e = threadIdx.x; e < N * N; e += kThreads) {
    const int x = e / N, y = e - x * N;
    W3[(size_t)x * ld + y] = Vs[e];
  }
  __syncthreads();
  cta_gemm<double, true, false>(N, N, N, W0, ld, W3, ld, W1, ld, S.gemm);
  cta_gemm<double, true, false>(N, N, N, W3, ld, W1, ld, W2, ld, S.gemm);
  const double dt = C.dtau;
  for (int e = threadIdx.x; e < N * N; e += kThreads) {
    const int a = e / N, b = e - a * N;
    const double la = ws[a], lb = ws[b];
    const double x = 0.5 * dt * (la - lb);
    const double shc = (x == 0.0) ? 1.0 : sinh(x) / x;
    W2[(size_t)a * ld + b] *= -dt * exp(-0.5 * dt * (la + lb)) * shc;
  }
  __syncthreads();
  cta_gemm<double, false, false>(N, N, N, W3, ld, W2, ld, W1, ld, S.gemm);
  cta_gemm<double, false, true>(N, N, N, W1, ld, W3, ld, W0, ld, S.gemm);
  double* out = gK + ((size_t)c * nfl + s) * N * N;
  for (int e = threadIdx.x; e < N * N; e += kThreads) {
    const int x = e / N, y = e - x * N;
    const double gxy = W0[(size_t)x * ld + y];
    out[e] = (x == y) ? gxy : gxy + W0[(size_t)y * ld + x];
  }
}

cudaError_t launch_logdet_grad(ChainDev* chains, int n_cfg, int nfl, const double* eigvec, const double* eigval,
                               double* gK, double* gU, double*, cudaStream_t st) {
  const size_t smem = get_smem_bytes();
  cudaError_t e = set_smem((const void*)logdet_grad_kernel, smem);
  if (e != cudaSuccess) return e;
  logdet_grad_kernel<<<n_cfg * nfl, kThreads, smem, st>>>(chains, n_cfg, eigvec, eigval, gK, gU);
  return cudaGetLastError();
}

}  // namespace dqmc
