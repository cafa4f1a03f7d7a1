// Adjoint of the energy estimator on fixed fields, with the time-displaced
// Green functions from the UDV chains.
#include "dqmc_device.cuh"

namespace dqmc {

// G(0) of every (configuration, flavor) into G0all [n_cfg][nfl][N][N] (FP64).
__global__ void __launch_bounds__(kThreads) green0_kernel(ChainDev* chains, int n_cfg, double* G0all) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nfl = chains[0].nfl;
  const int c = blockIdx.x / nfl, s = blockIdx.x % nfl;
  if (c >= n_cfg) return;
  ChainDev& C = chains[c];
  Smem S = carve_smem(smem_raw, C.ld, C.MV);
  double logdet;
  int sign;
  if (fill_left_chain(C, s, S, logdet, sign)) {
    if (threadIdx.x == 0) C.error = 1;
    return;
  }
  const double* Gf = wmat(C, s, 6);
  double* out = G0all + ((size_t)c * nfl + s) * C.N * C.N;
  for (int e = threadIdx.x; e < C.N * C.N; e += kThreads) {
    const int x = e / C.N, y = e - x * C.N;
    out[e] = Gf[(size_t)x * C.ld + y];
  }
  if (threadIdx.x == 0) { C.logdet[s] = logdet; C.fresh_sign[s] = sign; }
}

// Adjoint of the energy estimator E(G(0)) = Kin + Pot on fixed fields.  With
// Gamma = dE/dG (= -K^T - diag(U (1 - G^other_ii))), the implicit part is
//   sum_tau Tr[Z_tau dB_tau],  Z_tau = G(tau-1,0) Gamma^T G(0,tau),
// dB_tau = dE e^{V} + E e^{V} dV: hopping through sum_tau e^{V} Z_tau and the
// Frechet derivative of exp(-dtau K), coupling through (Z E e^{V})_ii dv_i/dU.
// G(tau,0) = B_tau G(tau-1,0) and G(0,tau) = G(0,tau-1) B_tau^-1 are wrapped
// between stabilisation points and recomputed from the chains at each one.
// Outputs per (configuration, flavor): gK [N][N] (explicit + implicit, pairs
// (x,y),(y,x) varied together), gU (implicit; flavor 0 adds the explicit
// sum (1-G_up)(1-G_dn)), eparts = (Kin_s, Part_s, Pot if flavor 0).
__global__ void __launch_bounds__(kThreads) energy_grad_kernel(ChainDev* chains, int n_cfg, const double* V,
                                                               const double* w, const double* G0all, double* ework_all,
                                                               double* gK, double* gU, double* eparts) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nfl = chains[0].nfl;
  const int c = blockIdx.x / nfl, s = blockIdx.x % nfl;
  if (c >= n_cfg) return;
  ChainDev& C = chains[c];
  Smem S = carve_smem(smem_raw, C.ld, C.MV);
  const int N = C.N, ld = C.ld, L = C.L, nw = C.nw, nst = L / nw;
  const size_t mat = (size_t)N * ld;
  double* ew = ework_all + ((size_t)c * nfl + s) * 6 * mat;
  double* Gam = ew;
  double* Gt0 = ew + mat;
  double* G0t = ew + 2 * mat;
  double* SE = ew + 3 * mat;
  double* T1 = ew + 4 * mat;
  double* T2 = ew + 5 * mat;
  double logdet;
  int sign;
  if (fill_left_chain(C, s, S, logdet, sign)) {  // storage slots: left chains; W6 = G(0)
    if (threadIdx.x == 0) C.error = 1;
    return;
  }
  const double* G0 = G0all + ((size_t)c * nfl + s) * N * N;
  const double* G0o = G0all + ((size_t)c * nfl + (nfl == 2 ? 1 - s : s)) * N * N;
  const double* K = C.K[s];
  double kin = 0.0, part = 0.0, pot = 0.0, potU = 0.0;
  for (int e = threadIdx.x; e < N * N; e += kThreads) {
    const int x = e / N, y = e - x * N;
    double g = -K[(size_t)x * ld + y];
    if (x == y && nfl == 2) g -= C.U * (1.0 - G0o[x * N + x]);
    Gam[(size_t)x * ld + y] = g;
    Gt0[(size_t)x * ld + y] = G0[e];                                  // G(0,0) = G(0)
    G0t[(size_t)x * ld + y] = -((x == y ? 1.0 : 0.0) - G0[e]);       // G(0,0^+) = -(1 - G(0))
    SE[(size_t)x * ld + y] = 0.0;
    kin += K[(size_t)x * ld + y] * ((x == y ? 1.0 : 0.0) - G0[y * N + x]);
  }
  for (int x = threadIdx.x; x < N; x += kThreads) {
    part += 1.0 - G0[x * N + x];
    if (nfl == 2) {
      const double t = (1.0 - G0[x * N + x]) * (1.0 - G0o[x * N + x]);
      potU += t;
      pot += C.U * t;
    }
  }
  kin = block_sum(kin, S.red);
  part = block_sum(part, S.red);
  pot = block_sum(pot, S.red);
  potU = block_sum(potU, S.red);
  double gu = 0.0;
  double* Z = wmat(C, s, 9);
  for (int tau = 1; tau <= L; ++tau) {
    slice_potential_global(C, s, tau, S.v);
    for (int x = threadIdx.x; x < N; x += kThreads) {
      S.ev[x] = exp(S.v[x]);
      S.hv[x] = exp(-S.v[x]);
    }
    __syncthreads();
    const bool stab = (tau % nw == 0);
    if (stab) {
      const int j = tau / nw;
      const UDV src = (j == 1) ? ident_udv(C) : slot_udv(C, s, j - 1);
      const int dq = chain_step(C, s, (j - 1) * nw, j * nw, false, src, S);
      const UDV Lf = (j == nst) ? ident_udv(C) : slot_udv(C, s, j);
      if (displaced_from_udv(C, s, work_udv(C, s, dq), Lf, T2, G0t, S)) {
        if (threadIdx.x == 0) C.error = 1;
        return;
      }
      copy_udv_to_slot(C, s, j, dq);
    } else {
      // G(0,tau) = G(0,tau-1) e^{-V} E^-1
      for (int e = threadIdx.x; e < N * N; e += kThreads) {
        const int x = e / N, y = e - x * N;
        G0t[(size_t)x * ld + y] *= S.hv[y];
      }
      __syncthreads();
      cta_gemm<double, false, false>(N, N, N, G0t, ld, C.Einv[s], ld, T1, ld, S.gemm);
      double* t_ = G0t; G0t = T1; T1 = t_;
    }
    // Z = G(tau-1,0) Gamma^T G(0,tau)
    cta_gemm<double, false, false>(N, N, N, Gt0, ld, Gam, ld, T1, ld, S.gemm);
    cta_gemm<double, false, false>(N, N, N, T1, ld, G0t, ld, Z, ld, S.gemm);
    for (int e = threadIdx.x; e < N * N; e += kThreads) {
      const int x = e / N, y = e - x * N;
      SE[(size_t)x * ld + y] += S.ev[x] * Z[(size_t)x * ld + y];
    }
    for (int k = threadIdx.x; k < C.MV; k += kThreads) {
      const int i = C.site[k];
      double acc = 0.0;
      for (int q = 0; q < N; ++q) acc = fma(Z[(size_t)i * ld + q], C.E[s][(size_t)q * ld + i], acc);
      gu += acc * S.ev[i] * C.vsign[s * C.MV + k] *
            coupling_dU(C.ft, C.dtau, C.U, C.cscale, C.fields[(size_t)(tau - 1) * C.MV + k]);
    }
    __syncthreads();
    // advance G(tau-1,0) -> G(tau,0)
    if (stab) {
      double* t_ = Gt0; Gt0 = T2; T2 = t_;
    } else {
      for (int e = threadIdx.x; e < N * N; e += kThreads) {
        const int x = e / N, y = e - x * N;
        Gt0[(size_t)x * ld + y] *= S.ev[x];
      }
      __syncthreads();
      cta_gemm<double, false, false>(N, N, N, C.E[s], ld, Gt0, ld, T1, ld, S.gemm);
      double* t_ = Gt0; Gt0 = T1; T1 = t_;
    }
  }
  gu = block_sum(gu, S.red);
  // implicit hopping part: V [F o (V^T SE^T V)] V^T
  double* W0 = wmat(C, s, 0);
  double* W1 = wmat(C, s, 1);
  double* W2 = wmat(C, s, 2);
  double* W3 = wmat(C, s, 3);
  const double* Vs = V + (size_t)s * N * N;
  const double* ws = w + (size_t)s * N;
  for (int e = threadIdx.x; e < N * N; e += kThreads) {
    const int x = e / N, y = e - x * N;
    W3[(size_t)x * ld + y] = Vs[e];
  }
  __syncthreads();
  cta_gemm<double, true, false>(N, N, N, SE, ld, W3, ld, W1, ld, S.gemm);
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
    const double ex = (x == y ? 1.0 : 0.0) - G0[y * N + x];
    const double exT = (x == y ? 1.0 : 0.0) - G0[x * N + y];
    out[e] = (x == y) ? W0[(size_t)x * ld + y] + ex
                      : W0[(size_t)x * ld + y] + W0[(size_t)y * ld + x] + ex + exT;
  }
  if (threadIdx.x == 0) {
    gU[(size_t)c * nfl + s] = gu + (s == 0 ? potU : 0.0);
    double* ep = eparts + ((size_t)c * nfl + s) * 3;
    ep[0] = kin;
    ep[1] = part;
    ep[2] = (s == 0) ? pot : 0.0;
  }
}

cudaError_t launch_energy_grad(ChainDev* chains, int n_cfg, int nfl, const double* eigvec, const double* eigval,
                               double* G0all, double* ework, double* gK, double* gU, double* eparts,
                               cudaStream_t st) {
  const size_t smem = get_smem_bytes();
  cudaError_t e = set_smem((const void*)green0_kernel, smem);
  if (e != cudaSuccess) return e;
  e = set_smem((const void*)energy_grad_kernel, smem);
  if (e != cudaSuccess) return e;
  green0_kernel<<<n_cfg * nfl, kThreads, smem, st>>>(chains, n_cfg, G0all);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  energy_grad_kernel<<<n_cfg * nfl, kThreads, smem, st>>>(chains, n_cfg, eigvec, eigval, G0all, ework, gK, gU,
                                                          eparts);
  return cudaGetLastError();
}

}  // namespace dqmc
