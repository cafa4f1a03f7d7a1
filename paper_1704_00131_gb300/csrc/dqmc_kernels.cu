// GB300 (sm_103a) kernels of the DQMC method that do not depend on the working
// precision and are light to compile: Philox initial fields, statistics reset,
// the equal-time correlation functions, and the dispatch to the per-precision
// sweep units.  Elsewhere: the adjoints (dqmc_grad_logdet.cu,
// dqmc_grad_energy.cu), the time-displaced measurement (dqmc_tau.cu), the
// allocation-free entry point (dqmc_noalloc.cu), the device building blocks
// (dqmc_device.cuh).
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

// After an initial fill: sign of the weight = product of the flavors' fresh signs.
__global__ void finalize_init_kernel(ChainDev* chains, int n_chains) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_chains) return;
  ChainDev& C = chains[c];
  int sg = 1;
  for (int s = 0; s < C.nfl; ++s) sg *= C.fresh_sign[s];
  C.sign = sg;
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

size_t smem_tail(size_t ab_bytes, int umma) { return smem_tail_bytes(ab_bytes, umma != 0); }

size_t plane_bytes(int N, int kmax) { return umma_plane_elems(N, kmax) * sizeof(__nv_bfloat16); }

// Digit planes and row exponents of a constant operand of the split products
// (one CTA): the left factor's rows (tiles of kUmmaM) or the right factor's
// columns (tiles of kUmmaNT), laid out as gemm_umma stages them.
__global__ void __launch_bounds__(kThreads) const_planes_kernel(const dd* X, int N, int ld, int right, int tr,
                                                                __nv_bfloat16* P, int* ex) {
  const int rows = right ? kUmmaNT : kUmmaM;
  const int Rp = umma_pad(N, rows), Kp = umma_pad(N, kUmmaK);
  // logical row r of the operand: row r of X, or column r (transpose / right factor)
  const bool colwise = right ? !tr : tr;
  if (colwise) umma_row_exponents<true>(N, N, X, ld, Rp, ex);
  else umma_row_exponents<false>(N, N, X, ld, Rp, ex);
  __syncthreads();
  if (colwise) umma_planes<true>(N, N, X, ld, Rp, Kp, rows, ex, P);
  else umma_planes<false>(N, N, X, ld, Rp, Kp, rows, ex, P);
}

size_t const_plane_bytes(int N, int right) {
  return (size_t)kUmmaDig * umma_pad(N, right ? kUmmaNT : kUmmaM) * umma_pad(N, kUmmaK) * sizeof(__nv_bfloat16);
}
int const_plane_exps(int N, int right) { return umma_pad(N, right ? kUmmaNT : kUmmaM); }

cudaError_t launch_const_planes(const void* X, int N, int ld, int right, int tr, void* planes, int* ex,
                                cudaStream_t st) {
  const_planes_kernel<<<1, kThreads, 0, st>>>((const dd*)X, N, ld, right, tr, (__nv_bfloat16*)planes, ex);
  return cudaGetLastError();
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
  if (precision == 3) return launch_fresh_green_mixed_tc(chains, n_chains, nfl, g_smem_bytes, mode, out, out_chain, st);
  return launch_fresh_green_mixed(chains, n_chains, nfl, g_smem_bytes, mode, out, out_chain, st);
}

cudaError_t launch_green_tau(ChainDev* chains, int chain, int nfl, int precision, int tau, double* out,
                             cudaStream_t st) {
  if (precision == 0) return launch_green_tau_fp64(chains, chain, nfl, g_smem_bytes, tau, out, st);
  if (precision == 1) return launch_green_tau_fp32(chains, chain, nfl, g_smem_bytes, tau, out, st);
  if (precision == 3) return launch_green_tau_mixed_tc(chains, chain, nfl, g_smem_bytes, tau, out, st);
  return launch_green_tau_mixed(chains, chain, nfl, g_smem_bytes, tau, out, st);
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
size_t get_smem_bytes() { return g_smem_bytes; }

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
  if (precision == 3) return launch_sweep_mixed_tc(chains, p, nfl, smem, st);
  return launch_sweep_mixed(chains, p, nfl, smem, st);
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

}  // namespace dqmc
