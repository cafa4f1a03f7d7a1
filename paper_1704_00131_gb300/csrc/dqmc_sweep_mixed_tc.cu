// Sweep and fresh-G kernels instantiated for the float-pair working Green function
// with the split tensor-core products (DQMC_PREC_MIXED_TC; chains below the
// tensor-core size threshold use the SIMT products at run time).
#define DQMC_WITH_UMMA 1
#include "dqmc_device.cuh"

namespace dqmc {

cudaError_t launch_sweep_mixed_tc(ChainDev* chains, const SweepParams& p, int nfl, size_t smem, cudaStream_t st) {
  return launch_sweep_t<dd>(chains, p, nfl, smem, st);
}

cudaError_t launch_fresh_green_mixed_tc(ChainDev* chains, int n_chains, int nfl, size_t smem, int mode, double* out,
                                     int out_chain, cudaStream_t st) {
  return launch_fresh_green_t<dd>(chains, n_chains, nfl, smem, mode, out, out_chain, st);
}

cudaError_t launch_green_tau_mixed_tc(ChainDev* chains, int chain, int nfl, size_t smem, int tau, double* out,
                                  cudaStream_t st) {
  return launch_green_tau_t<dd>(chains, chain, nfl, smem, tau, out, st);
}

}  // namespace dqmc
