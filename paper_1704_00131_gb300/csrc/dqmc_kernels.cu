// GB300 (sm_103a) kernels of the DQMC method that do not depend on the working
// precision: Philox initial fields, statistics reset, the log-det and energy
// adjoints (with the time-displaced Green functions), and the dispatch to the
// per-precision sweep units.  The device building blocks are in dqmc_device.cuh.
#include "dqmc_device.cuh"

namespace dqmc {

__global__ void init_fields_kernel(ChainDev* chains, int n_chains, uint64_t seed) {
  const int c = blockIdx.x;
  if (c >= n_chains) return;
  const ChainDev& C = chains[c];
  for (int e = threadIdx.x; e < C.L * C.MV; e += kThreads) {
    const int t = e / C.MV, k = e - t * C.MV;
    uint32_t ctr[4] = {0xFFFFFFFFu, (uint32_t)(t + 1), (uint32_t)k, 0xFFFFFFFFu};
    philox4x32_10(ctr, (uint32_t)seed, (uint32_t)(seed >> 32) ^ C.chain_id);
    const double u = uniform53(ctr[0], ctr[1]);
    int8_t f;
    if (C.ft == 1) {
      f = u < 0.5 ? -1 : 1;
    } else {
      int idx = (int)floor(4.0 * u);
      idx = idx > 3 ? 3 : idx;
      const int8_t vals[4] = {-2, -1, 1, 2};
      f = vals[idx];
    }
    C.fields[e] = f;
  }
}

__global__ void reset_stats_kernel(ChainDev* chains, int n_chains) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_chains) return;
  ChainDev& C = chains[c];
  for (int s = 0; s < kMaxFlavors; ++s) {
    C.prec_sum[s] = 0.0;
    C.prec_max[s] = 0.0;
    for (int q = 0; q < 4; ++q) C.cyc[s][q] = 0;
    for (int q = 0; q < 8; ++q) C.cycd[s][q] = 0;
  }
  C.phase_max = 0.0;
  C.prec_events = 0;
  C.proposals = 0;
  C.accepted = 0;
  C.sweep_sign_sum = 0.0;
}

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

// After an initial fill: sign of the weight = product of the flavors' fresh signs.
__global__ void finalize_init_kernel(ChainDev* chains, int n_chains) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_chains) return;
  ChainDev& C = chains[c];
  int sg = 1;
  for (int s = 0; s < C.nfl; ++s) sg *= C.fresh_sign[s];
  C.sign = sg;
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

// Time-displaced measurement of every chain's current configuration (the tau
// measurement at the end of a sweep, Algorithm 1; ObserT of Sec. 5.2).  The
// storage slots hold the left chains B(beta, j n_wrap)^T and are only read;
// the right chain B(tau,0) is built in the work UDV (chain steps in place).
// From G(0) = (1 + B(beta,0))^-1 the three functions are wrapped slice by slice,
//   G(tau,0)   = B_tau G(tau-1,0)
//   G(0,tau)   = G(0,tau-1) B_tau^-1
//   G(tau,tau) = B_tau G(tau-1,tau-1) B_tau^-1,
// and at every stabilisation point tau = j n_wrap replaced by the stable
// recompute from the chains; the largest and mean element difference of the
// wrapped G(tau,0), G(0,tau) against the recompute is the "Precision tau"
// monitor (Sec. 2.3).  Per tau the flavor's CTA writes
//   a = sum_x G(tau,0)_xx,  c = -sum_xy ph_x ph_y G(0,tau)_yx G(tau,0)_xy,
//   p = sum_x ph_x (1 - G(tau,tau)_xx).
// Buffers: tw [n_chains][nfl][4][N][ld] (G(tau,0), G(0,tau), G(tau,tau), temp);
// obs [n_chains][n_tau+1][nfl][3]; prec [n_chains][nfl][3] = (sum of element
// means, max, events); sign [n_chains][nfl].
__global__ void __launch_bounds__(kThreads) tau_measure_kernel(ChainDev* chains, int n_chains, int n_tau,
                                                               const double* phase, int phase_ld, double* tw_all,
                                                               size_t tw_stride, double* obs, double* prec,
                                                               int* sign_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nfl = chains[0].nfl;
  const int c = blockIdx.x / nfl, s = blockIdx.x % nfl;
  if (c >= n_chains) return;
  ChainDev& C = chains[c];
  Smem S = carve_smem(smem_raw, C.ld, C.MV);
  const int N = C.N, ld = C.ld, nw = C.nw, nst = C.L / nw;
  const int ntc = n_tau < C.L ? n_tau : C.L;
  const size_t mat = (size_t)N * ld;
  double* tw = tw_all + ((size_t)c * nfl + s) * tw_stride;
  double* Gt0 = tw;
  double* G0t = tw + mat;
  double* Gtt = tw + 2 * mat;
  double* T1 = tw + 3 * mat;
  const double* ph = phase + (size_t)c * phase_ld;
  double* o = obs + (size_t)c * (n_tau + 1) * nfl * 3;
  for (int e = threadIdx.x; e < (n_tau + 1) * nfl * 3; e += kThreads)
    if (e / 3 % nfl == s) o[e] = 0.0;
  // tau = 0 from the stored left chain
  double logdet;
  int sg;
  double* Gf = wmat(C, s, 6);
  if (green_from_udv(C, s, ident_udv(C), slot_udv(C, s, 0), Gf, logdet, sg, S)) {
    if (threadIdx.x == 0) C.error = 1;
    return;
  }
  if (threadIdx.x == 0) sign_out[(size_t)c * nfl + s] = sg;
  for (int e = threadIdx.x; e < N * N; e += kThreads) {
    const int x = e / N, y = e - x * N;
    const double g = Gf[(size_t)x * ld + y];
    Gt0[(size_t)x * ld + y] = g;
    Gtt[(size_t)x * ld + y] = g;
    G0t[(size_t)x * ld + y] = g - (x == y ? 1.0 : 0.0);
  }
  __syncthreads();
  double ev_sum = 0.0, ev_max = 0.0;
  int events = 0, dq = 1;
  for (int tau = 0; tau <= ntc; ++tau) {
    if (tau > 0) {
      slice_potential_global(C, s, tau, S.v);
      for (int x = threadIdx.x; x < N; x += kThreads) {
        S.ev[x] = exp(S.v[x]);
        S.hv[x] = exp(-S.v[x]);
      }
      __syncthreads();
      for (int e = threadIdx.x; e < N * N; e += kThreads) {
        const int x = e / N, y = e - x * N;
        Gt0[(size_t)x * ld + y] *= S.ev[x];
        G0t[(size_t)x * ld + y] *= S.hv[y];
        Gtt[(size_t)x * ld + y] *= S.ev[x] * S.hv[y];
      }
      __syncthreads();
      cta_gemm<double, false, false>(N, N, N, C.E[s], ld, Gt0, ld, T1, ld, S.gemm);
      { double* t_ = Gt0; Gt0 = T1; T1 = t_; }
      cta_gemm<double, false, false>(N, N, N, G0t, ld, C.Einv[s], ld, T1, ld, S.gemm);
      { double* t_ = G0t; G0t = T1; T1 = t_; }
      cta_gemm<double, false, false>(N, N, N, C.E[s], ld, Gtt, ld, T1, ld, S.gemm);
      cta_gemm<double, false, false>(N, N, N, T1, ld, C.Einv[s], ld, Gtt, ld, S.gemm);
      if (tau % nw == 0) {
        const int j = tau / nw;
        dq = chain_step(C, s, (j - 1) * nw, j * nw, false, (j == 1) ? ident_udv(C) : work_udv(C, s, dq), S);
        const UDV R = work_udv(C, s, dq);
        const UDV Lf = (j == nst) ? ident_udv(C) : slot_udv(C, s, j);
        double* Ft0 = wmat(C, s, 3);
        double* F0t = wmat(C, s, 4);
        int bad = displaced_from_udv(C, s, R, Lf, Ft0, F0t, S);
        if (!bad) bad = green_from_udv(C, s, R, Lf, Gf, logdet, sg, S);
        if (bad) {
          if (threadIdx.x == 0) C.error = 1;
          return;
        }
        double mx = 0.0, sm = 0.0;
        for (int e = threadIdx.x; e < N * N; e += kThreads) {
          const int x = e / N, y = e - x * N;
          const size_t q = (size_t)x * ld + y;
          const double d1 = fabs(Ft0[q] - Gt0[q]), d2 = fabs(F0t[q] - G0t[q]);
          mx = fmax(mx, fmax(d1, d2));
          sm += d1 + d2;
          Gt0[q] = Ft0[q];
          G0t[q] = F0t[q];
          Gtt[q] = Gf[q];
        }
        mx = block_max(mx, S.red);
        sm = block_sum(sm, S.red);
        ev_max = fmax(ev_max, mx);
        ev_sum += sm / (2.0 * N * N);
        ++events;
      }
    }
    double a = 0.0, cc = 0.0, p = 0.0;
    for (int x = threadIdx.x; x < N; x += kThreads) {
      a += Gt0[(size_t)x * ld + x];
      p += ph[x] * (1.0 - Gtt[(size_t)x * ld + x]);
    }
    for (int e = threadIdx.x; e < N * N; e += kThreads) {
      const int x = e / N, y = e - x * N;
      cc -= ph[x] * ph[y] * G0t[(size_t)y * ld + x] * Gt0[(size_t)x * ld + y];
    }
    a = block_sum(a, S.red);
    cc = block_sum(cc, S.red);
    p = block_sum(p, S.red);
    if (threadIdx.x == 0) {
      double* ot = o + ((size_t)tau * nfl + s) * 3;
      ot[0] = a;
      ot[1] = cc;
      ot[2] = p;
    }
  }
  if (threadIdx.x == 0) {
    double* pr = prec + ((size_t)c * nfl + s) * 3;
    pr[0] = ev_sum;
    pr[1] = ev_max;
    pr[2] = (double)events;
  }
}

// Equal-time correlation functions of every chain's current configuration
// (equal-time observables of Sec. 5.2 / 6, spin-z decoupling, flavor 0 up and
// 1 down), from the working G(0) of both flavors.  Wick's theorem per
// configuration (flavors independent), with X^s_xy = (delta_xy - G^s_yx) G^s_xy:
//   <S^z_x S^z_y> = [m_x m_y + X^0_xy + X^1_xy] / 4,  m_x = G^1_xx - G^0_xx
//   <n_x n_y>     = rho_x rho_y + X^0_xy + X^1_xy,    rho_x = 2 - G^0_xx - G^1_xx
//   <S^+_x S^-_y> = (delta_xy - G^0_yx) G^1_xy
//   sum_s <c^+_xs c_ys> = sum_s (delta_xy - G^s_yx)
// summed over the pairs of each class.  One thread per class walks the class's
// pairs in a fixed order (deterministic sums).  csr: per chain, class offsets
// [n_class + 1] into the pair list (x * N + y); out [n_chains][max_class][4].
template <typename Real>
__global__ void corr_kernel(ChainDev* chains, int n_chains, const int* csr_all, const int* pairs_all,
                            const int* chain_csr, const int* chain_pairs, const int* chain_ncls, int max_cls,
                            double* out) {
  const int c = blockIdx.x;
  if (c >= n_chains) return;
  const ChainDev& C = chains[c];
  const int N = C.N, ld = C.ld, ncls = chain_ncls[c];
  const int* off = csr_all + chain_csr[c];
  const int* pairs = pairs_all + chain_pairs[c];
  const Real* G0 = (const Real*)C.G[0];
  const Real* G1 = (const Real*)C.G[1];
  double* o = out + (size_t)c * max_cls * 4;
  for (int k = threadIdx.x; k < max_cls; k += blockDim.x) {
    double zz = 0.0, nn = 0.0, pm = 0.0, gf = 0.0;
    if (k < ncls) {
      for (int p = off[k]; p < off[k + 1]; ++p) {
        const int x = pairs[p] / N, y = pairs[p] - (pairs[p] / N) * N;
        const double dxy = (x == y) ? 1.0 : 0.0;
        const double g0xx = to_d(G0[(size_t)x * ld + x]), g1xx = to_d(G1[(size_t)x * ld + x]);
        const double g0yy = to_d(G0[(size_t)y * ld + y]), g1yy = to_d(G1[(size_t)y * ld + y]);
        const double g0xy = to_d(G0[(size_t)x * ld + y]), g0yx = to_d(G0[(size_t)y * ld + x]);
        const double g1xy = to_d(G1[(size_t)x * ld + y]), g1yx = to_d(G1[(size_t)y * ld + x]);
        const double X0 = (dxy - g0yx) * g0xy, X1 = (dxy - g1yx) * g1xy;
        const double mx = g1xx - g0xx, my = g1yy - g0yy;
        const double rx = 2.0 - g0xx - g1xx, ry = 2.0 - g0yy - g1yy;
        zz += 0.25 * (mx * my + X0 + X1);
        nn += rx * ry + X0 + X1;
        pm += (dxy - g0yx) * g1xy;
        gf += (dxy - g0yx) + (dxy - g1yx);
      }
    }
    o[k * 4 + 0] = zz;
    o[k * 4 + 1] = nn;
    o[k * 4 + 2] = pm;
    o[k * 4 + 3] = gf;
  }
}

// --------------------------------------------------------------------------
// Launchers.
// --------------------------------------------------------------------------
size_t sweep_smem_bytes(int maxN, int maxld, int maxMV, int delay_k, int precision) {
  (void)maxN; (void)delay_k; (void)precision;
  return smem_bytes_for(maxld, maxMV);
}

cudaError_t launch_init_fields(ChainDev* chains, int n_chains, uint64_t seed, int, int, cudaStream_t st) {
  init_fields_kernel<<<n_chains, kThreads, 0, st>>>(chains, n_chains, seed);
  return cudaGetLastError();
}

static size_t g_smem_bytes = 0;

cudaError_t launch_fresh_green(ChainDev* chains, int n_chains, int nfl, int precision, int write_working,
                               double* out, int out_chain, cudaStream_t st) {
  const int mode = write_working ? 0 : 1;
  if (precision == 0) return launch_fresh_green_fp64(chains, n_chains, nfl, g_smem_bytes, mode, out, out_chain, st);
  if (precision == 1) return launch_fresh_green_fp32(chains, n_chains, nfl, g_smem_bytes, mode, out, out_chain, st);
  return launch_fresh_green_mixed(chains, n_chains, nfl, g_smem_bytes, mode, out, out_chain, st);
}

cudaError_t launch_copy_green(ChainDev* chains, int chain, int flavor, int precision, double* out,
                              cudaStream_t st) {
  if (precision == 0)
    copy_green_kernel<double><<<16, 256, 0, st>>>(chains, chain, flavor, out);
  else if (precision == 1)
    copy_green_kernel<float><<<16, 256, 0, st>>>(chains, chain, flavor, out);
  else
    copy_green_kernel<dd><<<16, 256, 0, st>>>(chains, chain, flavor, out);
  return cudaGetLastError();
}

void set_smem_bytes(size_t b) { g_smem_bytes = b; }

cudaError_t launch_finalize_init(ChainDev* chains, int n_chains, cudaStream_t st) {
  finalize_init_kernel<<<(n_chains + 127) / 128, 128, 0, st>>>(chains, n_chains);
  return cudaGetLastError();
}

cudaError_t launch_reset_stats(ChainDev* chains, int n_chains, cudaStream_t st) {
  reset_stats_kernel<<<(n_chains + 127) / 128, 128, 0, st>>>(chains, n_chains);
  return cudaGetLastError();
}

cudaError_t launch_sweep(ChainDev* chains, const SweepParams& p, int nfl, int precision, size_t smem,
                         cudaStream_t st) {
  if (precision == 0) return launch_sweep_fp64(chains, p, nfl, smem, st);
  if (precision == 1) return launch_sweep_fp32(chains, p, nfl, smem, st);
  return launch_sweep_mixed(chains, p, nfl, smem, st);
}

cudaError_t launch_energy_grad(ChainDev* chains, int n_cfg, int nfl, const double* eigvec, const double* eigval,
                               double* G0all, double* ework, double* gK, double* gU, double* eparts,
                               cudaStream_t st) {
  const size_t smem = g_smem_bytes;
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

cudaError_t launch_tau_measure(ChainDev* chains, int n_chains, int nfl, int n_tau, const double* phase,
                               int phase_ld, double* tw, size_t tw_stride, double* obs, double* prec, int* sign,
                               cudaStream_t st) {
  const size_t smem = g_smem_bytes;
  cudaError_t e = set_smem((const void*)tau_measure_kernel, smem);
  if (e != cudaSuccess) return e;
  tau_measure_kernel<<<n_chains * nfl, kThreads, smem, st>>>(chains, n_chains, n_tau, phase, phase_ld, tw,
                                                             tw_stride, obs, prec, sign);
  return cudaGetLastError();
}

cudaError_t launch_corr(ChainDev* chains, int n_chains, int precision, const int* csr_all, const int* pairs_all,
                        const int* chain_csr, const int* chain_pairs, const int* chain_ncls, int max_cls,
                        double* out, cudaStream_t st) {
  if (precision == 0)
    corr_kernel<double><<<n_chains, 128, 0, st>>>(chains, n_chains, csr_all, pairs_all, chain_csr, chain_pairs,
                                                  chain_ncls, max_cls, out);
  else if (precision == 1)
    corr_kernel<float><<<n_chains, 128, 0, st>>>(chains, n_chains, csr_all, pairs_all, chain_csr, chain_pairs,
                                                 chain_ncls, max_cls, out);
  else
    corr_kernel<dd><<<n_chains, 128, 0, st>>>(chains, n_chains, csr_all, pairs_all, chain_csr, chain_pairs,
                                              chain_ncls, max_cls, out);
  return cudaGetLastError();
}

cudaError_t launch_logdet_grad(ChainDev* chains, int n_cfg, int nfl, const double* eigvec, const double* eigval,
                               double* gK, double* gU, double*, cudaStream_t st) {
  const size_t smem = g_smem_bytes;
  cudaError_t e = set_smem((const void*)logdet_grad_kernel, smem);
  if (e != cudaSuccess) return e;
  logdet_grad_kernel<<<n_cfg * nfl, kThreads, smem, st>>>(chains, n_cfg, eigvec, eigval, gK, gU);
  return cudaGetLastError();
}

}  // namespace dqmc

// ===========================================================================
// Allocation-free variant of the fresh G(0) computation.
//
// For callers that cannot allocate device memory (a host process running under
// a memory manager that owns every device allocation, or code that may not
// call cudaMalloc at the point where it needs G), this entry point computes
// G^s(0) = (1 + B^s(beta,0))^-1 from caller-owned device inputs, with all of
// its scratch in one file-scope device array of fixed size.  It keeps a
// running left UDV chain instead of the per-slot storage of the sweep, so the
// scratch does not grow with L.
// ===========================================================================
namespace {

constexpr int kNoAllocMaxN = 64;         // largest lattice the scratch array holds
constexpr int kNoAllocMaxFlavors = 2;
// per flavor: workspace (kWorkMats matrices + 8 vectors), one running UDV
// (Q, T, D), an identity UDV and the integer pivots, all with ld = N
constexpr size_t kNoAllocPerFlavor =
    (size_t)dqmc::kWorkMats * kNoAllocMaxN * kNoAllocMaxN + 8 * kNoAllocMaxN +
    2 * (2 * (size_t)kNoAllocMaxN * kNoAllocMaxN + kNoAllocMaxN) + 2 * kNoAllocMaxN;
constexpr size_t kNoAllocDoubles = kNoAllocMaxFlavors * kNoAllocPerFlavor;

// Shared by every call on a device; every GPU that loads the library holds it
// (about 1 MiB) until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

constexpr int kMaxDevices = 64;
static double* g_noalloc_ptr[kMaxDevices] = {nullptr};

}  // namespace

namespace dqmc {

// Left chain from beta down to 0 kept in one running UDV (slot 0), then G(0).
__device__ int left_chain_running(const ChainDev& C, int s, Smem& S, double& logdet, int& sign) {
  const int nst = C.L / C.nw;
  for (int j = nst - 1; j >= 0; --j) {
    const UDV src = (j + 1 == nst) ? ident_udv(C) : slot_udv(C, s, 0);
    const int dq = chain_step(C, s, j * C.nw, (j + 1) * C.nw, true, src, S);
    copy_udv_to_slot(C, s, 0, dq);
  }
  return green_from_udv(C, s, ident_udv(C), slot_udv(C, s, 0), wmat(C, s, 6), logdet, sign, S);
}

__global__ void __launch_bounds__(kThreads) fresh_green_noalloc_kernel(ChainDev C, double* scratch,
                                                                       double* out, double* logdet_out,
                                                                       int* sign_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int s = blockIdx.x;
  const int N = C.N, ld = C.ld;
  // carve this flavor's part of the scratch array
  double* base = scratch + (size_t)s * kNoAllocPerFlavor;
  ChainDev Cl = C;
  Cl.work[s] = base;
  double* slot = base + (size_t)kWorkMats * N * ld + 8 * ld;
  double* ident = slot + 2 * (size_t)N * ld + ld;
  int* ibase = reinterpret_cast<int*>(ident + 2 * (size_t)N * ld + ld);
  Cl.slots[s] = slot;
  Cl.ident = ident;
  Cl.iwork[s] = ibase;             // perm [ld], piv [ld]
  Cl.slot_detq[s] = ibase + 2 * ld;
  // the array keeps the previous call's contents: rebuild the identity UDV
  for (int e = threadIdx.x; e < N * N; e += kThreads) {
    const int x = e / N, y = e - x * N;
    ident[(size_t)x * ld + y] = (x == y) ? 1.0 : 0.0;
    ident[(size_t)N * ld + (size_t)x * ld + y] = (x == y) ? 1.0 : 0.0;
  }
  for (int x = threadIdx.x; x < N; x += kThreads) ident[(size_t)2 * N * ld + x] = 1.0;
  __syncthreads();
  Smem S = carve_smem(smem_raw, ld, C.MV);
  double logdet = 0.0;
  int sign = 0;
  const int bad = left_chain_running(Cl, s, S, logdet, sign);
  const double* Gf = wmat(Cl, s, 6);
  for (int e = threadIdx.x; e < N * N; e += kThreads) {
    const int x = e / N, y = e - x * N;
    out[(size_t)s * N * N + e] = Gf[(size_t)x * ld + y];
  }
  if (threadIdx.x == 0) {
    if (logdet_out) logdet_out[s] = bad ? 0.0 : logdet;
    if (sign_out) sign_out[s] = bad ? 0 : sign;
  }
}

}  // namespace dqmc

extern "C" dqmc_status dqmc_green_fresh_noalloc(int32_t n_sites, int32_t n_flavors, const double* E_dev,
                                        int32_t n_vertices, const int32_t* vertex_site_dev,
                                        const double* vertex_sign_dev, double U, int32_t field_type, double dtau,
                                        int32_t L, int32_t n_wrap, const int8_t* fields_dev, double* G_out_dev,
                                        double* logdet_out_dev, int32_t* sign_out_dev, void* cuda_stream) {
  using namespace dqmc;
  if (n_sites < 1 || n_sites > kNoAllocMaxN || n_flavors < 1 || n_flavors > kNoAllocMaxFlavors ||
      n_vertices < 1 || n_vertices > n_sites || (field_type != 1 && field_type != 2) || !(dtau > 0.0) ||
      !(U >= 0.0) || L < 1 || n_wrap < 1 || L % n_wrap != 0 || !E_dev || !vertex_site_dev ||
      !vertex_sign_dev || !fields_dev || !G_out_dev)
    return DQMC_EINVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DQMC_ECUDA;
  if (!g_noalloc_ptr[dev]) {
    // once per device, with that device current: the device address of the array
    double* p = nullptr;
    if (cudaGetSymbolAddress((void**)&p, g_noalloc_scratch) != cudaSuccess || !p) return DQMC_ECUDA;
    g_noalloc_ptr[dev] = p;
  }
  ChainDev C{};
  C.N = n_sites;
  C.ld = n_sites;
  C.nfl = n_flavors;
  C.MV = n_vertices;
  C.L = L;
  C.nw = n_wrap;
  C.ft = field_type;
  C.dtau = dtau;
  C.U = U;
  C.cscale = (field_type == 1) ? std::acosh(std::exp(0.5 * dtau * U)) : std::sqrt(0.5 * dtau * U);
  for (int s = 0; s < n_flavors; ++s) C.E[s] = E_dev + (size_t)s * n_sites * n_sites;
  C.site = vertex_site_dev;
  C.vsign = vertex_sign_dev;
  C.fields = const_cast<int8_t*>(fields_dev);
  const size_t smem = smem_bytes_for(n_sites, n_vertices);
  if (cudaFuncSetAttribute((const void*)fresh_green_noalloc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess)
    return DQMC_ECUDA;
  fresh_green_noalloc_kernel<<<n_flavors, kThreads, smem, (cudaStream_t)cuda_stream>>>(
      C, g_noalloc_ptr[dev], G_out_dev, logdet_out_dev, sign_out_dev);
  return cudaGetLastError() == cudaSuccess ? DQMC_OK : DQMC_ECUDA;
}
