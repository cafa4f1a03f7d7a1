// Internal declarations shared by the host side (dqmc_api.cu) and the kernels
// (dqmc_kernels.cu) of the GB300 DQMC library.  Not part of the public C ABI.
#pragma once
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace dqmc {

constexpr int kThreads = 256;      // threads per CTA of every kernel
constexpr int kMaxFlavors = 2;
// Digit planes of the split tensor-core products: blocks of kPlaneDigits digits
// x rows x kPlaneK bf16 (rows: kPlaneRowsA for a left operand, kPlaneRowsB for
// a right one), one block per (tile, 16-wide K chunk), copied to shared memory
// by one tiled tensor copy each.
constexpr int kPlaneDigits = 7, kPlaneRowsA = 64, kPlaneRowsB = 48, kPlaneK = 16;

// Device-resident description and state of one Markov chain.  One CTA per
// (chain, flavor) works on it; the CTAs of a chain form one thread-block
// cluster.  All matrices are row-major with leading dimension `ld`.
struct ChainDev {
  // model
  int N, ld, nfl, MV, L, nw, ft;  // ft: 1 Ising, 2 four-valued HS
  double dtau, U, cscale;         // cscale = lambda (Ising) or g (HS4)
  const double* K[kMaxFlavors];   // hopping [N][ld]
  const double* E[kMaxFlavors];   // exp(-dtau K) [N][ld]
  const double* Einv[kMaxFlavors];
  const float* E32[kMaxFlavors];  // FP32 copies for the mixed path
  const float* Einv32[kMaxFlavors];
  const void* Edd[kMaxFlavors];   // float-float (hi, lo) copies for the mixed path
  const void* Einvdd[kMaxFlavors];
  const int* site;                // [MV]
  const double* vsign;            // [nfl][MV]
  const double* ident;            // identity UDV: Q=I [N][ld], T=I [N][ld], D=1 [ld]
  // state
  int8_t* fields;                 // [L][MV]
  void* G[kMaxFlavors];           // working G (Real) [N][ld]
  void* Gtmp[kMaxFlavors];        // Real [N][ld] scratch for the wraps
  void* dA[kMaxFlavors];          // Real [k][ld] delayed vectors a_m
  void* dB[kMaxFlavors];          // Real [k][ld] delayed vectors b_m
  double* slots[kMaxFlavors];     // FP64 [nst+1] x {Q [N][ld], T [N][ld], D [ld]}
  int* slot_detq[kMaxFlavors];    // [nst+1]
  double* work[kMaxFlavors];      // FP64 stabilisation workspace, kWorkMats matrices + vectors
  void* planes[kMaxFlavors];      // BF16 digit planes of the split tensor-core products (mixed path)
  // digit planes and row exponents of the constant split operands, prepared once
  // per model: kCpEA = E as left factor, kCpEtA = E^T left, kCpEiA = E^-1 left,
  // kCpEiB = E^-1 right, kCpEB = E right (null without tensor-core products)
  const void* cpl[kMaxFlavors][5];
  const int* cex[kMaxFlavors][5];
  // tensor maps (4D views [blocks][digits][rows][k] with a box of one block) of
  // the scratch planes as left [0] and right [1] operand, and of the constant
  // operands' planes
  CUtensorMap tm_pl[kMaxFlavors][2];
  CUtensorMap tm_cp[kMaxFlavors][5];
  int* iwork[kMaxFlavors];        // [2*ld]
  uint32_t chain_id;
  int sign;                       // sign of the current weight (written by rank 0)
  // statistics of the current dqmc_sweep call, per flavor
  double prec_sum[kMaxFlavors], prec_max[kMaxFlavors];
  double phase_max;
  int64_t prec_events;
  int64_t proposals, accepted;
  double sweep_sign_sum;
  // measurement accumulators (sign-weighted) kin, pot, part, ener
  double meas[4];
  double meas_sign;
  int64_t n_meas;
  // last fresh log|det| and sign per flavor (written by greens/init kernels)
  double logdet[kMaxFlavors];
  int fresh_sign[kMaxFlavors];
  int error;                      // bit 0: a numerical failure; bit 1: a bounded device wait gave up
  long long wait_cycles;          // SM cycles before a bounded device wait gives up
  int stab_svd;                   // stabilisation by one-sided Jacobi SVD instead of the pivoted QR (FP64)
  int test_stall;                 // test hook: tensor-core products wait on a barrier nothing arrives on
  int dd_tile;                    // register tile of the float-pair SIMT products (0 by padding, 3, 4)
  int wait_where[kMaxFlavors][6]; // first wait that gave up per flavor: kind (1 copy, 2 MMAs
                                  // before a refill, 3 MMAs before the epilogue, 4 / 5 copy / MMAs
                                  // at the end of a product; 9 a staging buffer not 128-byte
                                  // aligned for the tensor copies), chunk (stage for 4, 5), chunks,
                                  // product ordinal in the kernel, barrier word (low, high)
  // SM cycles spent per phase during the current dqmc_sweep call, per flavor:
  // 0 updates, 1 wraps (V and T), 2 stabilisation, 3 measurement
  int64_t cyc[kMaxFlavors][4];
  // finer split, per flavor: 0 ratio precompute, 1 acceptance scan (ratios,
  // cluster barrier, first acceptance), 2 update vectors, 3 flushes,
  // 4 B-chain products, 5 QR and Q, 6 T update, 7 stable G
  int64_t cycd[kMaxFlavors][8];
};

constexpr int kWorkMats = 10;     // N x ld FP64 matrices per flavor in `work`
enum { kCpEA = 0, kCpEtA = 1, kCpEiA = 2, kCpEiB = 3, kCpEB = 4 };

__host__ __device__ inline size_t slot_stride(int N, int ld) { return (size_t)2 * N * ld + ld; }
__host__ __device__ inline size_t work_elems(int N, int ld) { return (size_t)kWorkMats * N * ld + 8 * (size_t)ld; }

struct SweepParams {
  uint64_t seed;
  uint64_t sweep;        // Philox sweep counter of this sweep
  int delay_k;
  int measure, meas_first, meas_last;
  int n_chains;
  int ab_smem;           // delayed vectors in shared memory (else in the chain's arena)
  const int* order;      // chain index for cluster c (heavy chains first)
};

// launchers (dqmc_kernels.cu)
cudaError_t launch_init_fields(ChainDev* chains, int n_chains, uint64_t seed, int maxL, int maxMV,
                               cudaStream_t st);
cudaError_t launch_fresh_green(ChainDev* chains, int n_chains, int nfl, int precision, int write_working,
                               double* out, int out_chain, cudaStream_t st);
cudaError_t launch_sweep(ChainDev* chains, const SweepParams& p, int nfl, int precision, size_t smem,
                         cudaStream_t st);
size_t sweep_smem_bytes(int maxN, int maxld, int maxMV, int delay_k, int precision);
// bytes of the shared-memory region behind the base (delayed vectors and/or the
// staging buffers of the split tensor-core products)
size_t smem_tail(size_t ab_bytes, int umma);
// bytes of the BF16 digit planes of one CTA's split products up to N x N x kmax
size_t plane_bytes(int N, int kmax);
// digit planes of a constant N x N float-pair operand: as the left factor
// (right = 0; tr = 1 for its transpose) or as the right factor (right = 1);
// bytes of the planes and entries of the exponent vector
size_t const_plane_bytes(int N, int right);
int const_plane_exps(int N, int right);
cudaError_t launch_const_planes(const void* X, int N, int ld, int right, int tr, void* planes, int* ex,
                                cudaStream_t st);
cudaError_t launch_copy_green(ChainDev* chains, int chain, int flavor, int precision, double* out,
                              cudaStream_t st);
cudaError_t launch_green_tau(ChainDev* chains, int chain, int nfl, int precision, int tau, double* out,
                             cudaStream_t st);
void set_smem_bytes(size_t bytes);
cudaError_t launch_energy_grad(ChainDev* chains, int n_cfg, int nfl, const double* eigvec, const double* eigval,
                               double* G0all, double* ework, double* gK, double* gU, double* eparts,
                               cudaStream_t st);
cudaError_t launch_finalize_init(ChainDev* chains, int n_chains, cudaStream_t st);
cudaError_t launch_corr(ChainDev* chains, int n_chains, int precision, const int* csr_all, const int* pairs_all,
                        const int* chain_csr, const int* chain_pairs, const int* chain_ncls, int max_cls,
                        double* out, cudaStream_t st);
// Class lists and outputs of the time-displaced correlation functions (all
// null / 0 when only the sums of dqmc_measure_tau are wanted).
struct TauCorrArgs {
  const int* csr_all = nullptr;      // per model: class offsets [n_class + 1] into its pair list
  const int* pairs_all = nullptr;    // per model: pairs x * N + y sorted by class, then x, y
  const int* chain_csr = nullptr;    // [n_chains] offset of the chain's model in csr_all
  const int* chain_pairs = nullptr;  // [n_chains] offset of the chain's model in pairs_all
  const int* chain_ncls = nullptr;   // [n_chains] number of classes of the chain's model
  int max_cls = 0;
  double* part = nullptr;            // [n_chains][n_tau+1][nfl][max_cls][2]
  double* dens = nullptr;            // [n_chains][n_tau+1][nfl][dens_ld]
  int dens_ld = 0;
};

cudaError_t launch_tau_measure(ChainDev* chains, int n_chains, int nfl, int n_tau, const double* phase,
                               int phase_ld, double* tw, size_t tw_stride, double* obs, double* prec, int* sign,
                               const TauCorrArgs& tc, cudaStream_t st);
cudaError_t launch_tau_corr_combine(const ChainDev* chains, int n_chains, int n_tau, const TauCorrArgs& tc,
                                    double* out, cudaStream_t st);
cudaError_t launch_reset_stats(ChainDev* chains, int n_chains, cudaStream_t st);
cudaError_t launch_logdet_grad(ChainDev* chains, int n_cfg, int nfl, const double* eigvec,
                               const double* eigval, double* gK, double* gU, double* Sacc,
                               cudaStream_t st);

}  // namespace dqmc
