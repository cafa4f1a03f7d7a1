// Time-displaced measurement of the chains' current configurations.
#include "dqmc_device.cuh"

namespace dqmc {

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
//
// With class lists (tc.part != nullptr) the flavor's CTA also writes, per tau and
// per class k of the chain's model, the flavor's share of the time-displaced
// correlation functions (the lattice-resolved ObserT quantities, Sec. 5.2):
//   part[c][tau][s][k] = (sum_(x,y) in k G^s(tau,0)_xy,
//                         sum_(x,y) in k X^s_xy),  X^s_xy = -G^s(0,tau)_yx G^s(tau,0)_xy,
//   dens[c][tau][s][x] = 1 - G^s(tau,tau)_xx,
// one thread per class walking the class's pairs in a fixed order; the flavors
// are combined by tau_corr_combine_kernel.
__global__ void __launch_bounds__(kThreads) tau_measure_kernel(ChainDev* chains, int n_chains, int n_tau,
                                                               const double* phase, int phase_ld, double* tw_all,
                                                               size_t tw_stride, double* obs, double* prec,
                                                               int* sign_out, TauCorrArgs tc) {
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
    if (tc.part) {
      const int ncls = tc.chain_ncls[c];
      const int* off = tc.csr_all + tc.chain_csr[c];
      const int* pairs = tc.pairs_all + tc.chain_pairs[c];
      double* pt = tc.part + (((size_t)c * (n_tau + 1) + tau) * nfl + s) * tc.max_cls * 2;
      for (int k = threadIdx.x; k < tc.max_cls; k += kThreads) {
        double gs = 0.0, xs = 0.0;
        if (k < ncls)
          for (int q = off[k]; q < off[k + 1]; ++q) {
            const int x = pairs[q] / N, y = pairs[q] - (pairs[q] / N) * N;
            const double gt0 = Gt0[(size_t)x * ld + y];
            gs += gt0;
            xs -= G0t[(size_t)y * ld + x] * gt0;
          }
        pt[2 * k] = gs;
        pt[2 * k + 1] = xs;
      }
      double* dn = tc.dens + (((size_t)c * (n_tau + 1) + tau) * nfl + s) * tc.dens_ld;
      for (int x = threadIdx.x; x < N; x += kThreads) dn[x] = 1.0 - Gtt[(size_t)x * ld + x];
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

// Time-displaced correlation functions per class from the flavors' shares (two
// flavors, spin-z decoupling, flavor 0 up and 1 down; Wick's theorem per
// configuration with independent flavors), n^s_x(tau) = 1 - G^s(tau,tau)_xx:
//   out[c][tau][k][0] = sum_s sum_(x,y) in k G^s(tau,0)_xy          (sum_s <c_xs(tau) c^+_ys(0)>)
//   out[c][tau][k][1] = sum_(x,y) in k [(n^0_x(tau) - n^1_x(tau)) (n^0_y(0) - n^1_y(0)) + X^0_xy + X^1_xy] / 4
//                                                                    (<S^z_x(tau) S^z_y(0)>)
//   out[c][tau][k][2] = sum_(x,y) in k [(n^0_x(tau) + n^1_x(tau)) (n^0_y(0) + n^1_y(0)) + X^0_xy + X^1_xy]
//                                                                    (<n_x(tau) n_y(0)>)
// Rows tau > L_c and classes beyond the chain's model's count are 0.
__global__ void tau_corr_combine_kernel(const ChainDev* chains, int n_chains, int n_tau, TauCorrArgs tc,
                                        double* out) {
  const int c = blockIdx.x / (n_tau + 1), tau = blockIdx.x % (n_tau + 1);
  if (c >= n_chains) return;
  const ChainDev& C = chains[c];
  const int N = C.N, ncls = tc.chain_ncls[c];
  const int* off = tc.csr_all + tc.chain_csr[c];
  const int* pairs = tc.pairs_all + tc.chain_pairs[c];
  const double* pt = tc.part + ((size_t)c * (n_tau + 1) + tau) * 2 * tc.max_cls * 2;
  const double* dt = tc.dens + ((size_t)c * (n_tau + 1) + tau) * 2 * tc.dens_ld;
  const double* d0 = tc.dens + ((size_t)c * (n_tau + 1)) * 2 * tc.dens_ld;
  double* o = out + ((size_t)c * (n_tau + 1) + tau) * tc.max_cls * 3;
  const bool live = tau <= C.L;
  for (int k = threadIdx.x; k < tc.max_cls; k += blockDim.x) {
    double g = 0.0, zz = 0.0, nn = 0.0;
    if (live && k < ncls) {
      const double X = pt[2 * k + 1] + pt[2 * tc.max_cls + 2 * k + 1];
      g = pt[2 * k] + pt[2 * tc.max_cls + 2 * k];
      for (int q = off[k]; q < off[k + 1]; ++q) {
        const int x = pairs[q] / N, y = pairs[q] - (pairs[q] / N) * N;
        const double nxu = dt[x], nxd = dt[tc.dens_ld + x], nyu = d0[y], nyd = d0[tc.dens_ld + y];
        zz += (nxu - nxd) * (nyu - nyd);
        nn += (nxu + nxd) * (nyu + nyd);
      }
      zz = 0.25 * (zz + X);
      nn += X;
    }
    o[3 * k] = g;
    o[3 * k + 1] = zz;
    o[3 * k + 2] = nn;
  }
}

cudaError_t launch_tau_measure(ChainDev* chains, int n_chains, int nfl, int n_tau, const double* phase,
                               int phase_ld, double* tw, size_t tw_stride, double* obs, double* prec, int* sign,
                               const TauCorrArgs& tc, cudaStream_t st) {
  const size_t smem = get_smem_bytes();
  cudaError_t e = set_smem((const void*)tau_measure_kernel, smem);
  if (e != cudaSuccess) return e;
  tau_measure_kernel<<<n_chains * nfl, kThreads, smem, st>>>(chains, n_chains, n_tau, phase, phase_ld, tw,
                                                             tw_stride, obs, prec, sign, tc);
  return cudaGetLastError();
}

cudaError_t launch_tau_corr_combine(const ChainDev* chains, int n_chains, int n_tau, const TauCorrArgs& tc,
                                    double* out, cudaStream_t st) {
  tau_corr_combine_kernel<<<n_chains * (n_tau + 1), 128, 0, st>>>(chains, n_chains, n_tau, tc, out);
  return cudaGetLastError();
}

}  // namespace dqmc
