// Internal declarations of the SU(2) charge-decoupling path, shared by the
// host side (dqmc_su2_api.cu) and the kernels (dqmc_su2.cu).  Not part of the
// public C ABI.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace dqmc {

// Device-resident description and state of one Markov chain of the SU(2)
// decoupling (Sec. 6.1), optionally with Ising spins on bonds coupling to the
// hopping (the Hubbard-Ising model of Sec. 6).  One CTA works on it.  Complex
// matrices are double2 (re, im), row-major with leading dimension `ld` (in
// complex elements).
struct Su2Dev {
  // model: B_tau = E X_0 X_1 ... X_{nb-1} exp(V_tau), V_tau = diag(i g eta(l_tau,x)),
  // g = sqrt(dtau U / 2), X_b = exp(a0 s_b O_b) on the bond (bi[b], bj[b]),
  // O_b = |i><j| + |j><i|, a0 = -dtau xi
  int N, ld, L, nw;
  int nb, MV;             // bonds; vertices per slice MV = N + nb (fields [L][MV])
  double dtau, U, g;
  double a0;              // -dtau xi
  double lch, lsh, dJ;    // log cosh(dtau h), log sinh(dtau h), dtau J (bond spins' weight)
  const int* bi;          // [nb]
  const int* bj;          // [nb]
  const int* nbr_off;     // [nb + 1] CSR of the J pairs: bonds paired with b are
  const int* nbr;         //   nbr[nbr_off[b] .. nbr_off[b + 1])
  const double* K;        // hopping [N][ld] (real symmetric, -mu on the diagonal)
  const double* E;        // exp(-dtau K) [N][ld]
  const double* Einv;     // exp(+dtau K) [N][ld]
  const double2* ident;   // identity [N][ld] (Q and T of the empty chain)
  const double* ones;     // [ld] of 1 (its D)
  // state
  int8_t* fields;         // [L][MV]: per slice the four-valued l in {-2, -1, 1, 2} of the
                          // N sites, then the Ising spins +-1 of the nb bonds
  double2* G;             // working G [N][ld]
  double2* Gt;            // scratch of the wraps [N][ld]
  double2* slots;         // (L/nw + 1) x {Q [N][ld], T [N][ld]}
  double* slotD;          // (L/nw + 1) x D [ld]
  int* slot_detq;         // [L/nw + 1]: det Q = +-1 (product of Householder reflectors)
  double2* work;          // kSu2Mats complex matrices [N][ld], then kSu2ZVecs complex vectors [ld]
  double* dwork;          // kSu2DVecs real vectors [ld]
  int* iwork;             // [ld] pivot order
  uint32_t chain_id;
  double2 P;              // phase of e^{-S(C)}: exp(i (ph + 2 arg det(1 + B(beta,0)))), ph = -g sum eta
  double logabs, arg;     // log|det(1 + B(beta,0))| and its argument at the last fresh G
  // statistics of the current dqmc_su2_sweep call
  double prec_sum, prec_max, phase_max;
  int64_t prec_events, proposals, accepted;
  double sweep_sign_sum;
  // reweighted measurement sums: (re, im) of kin, pot, part, ener and of the bond
  // spins' (sum_b s_b)^2 / nb averaged over the slices; sum of signs; count
  double meas[10];
  double meas_sign;
  int64_t n_meas;
  int error;              // bit 0: a singular matrix in the stabilisation
};

constexpr int kSu2Mats = 12;  // complex N x ld work matrices per chain
constexpr int kSu2ZVecs = 4;  // complex work vectors per chain
constexpr int kSu2DVecs = 10; // real work vectors per chain

__host__ __device__ inline size_t su2_slot_elems(int N, int ld) { return (size_t)2 * N * ld; }
__host__ __device__ inline size_t su2_work_elems(int N, int ld) {
  return (size_t)kSu2Mats * N * ld + (size_t)kSu2ZVecs * ld;
}

struct Su2SweepParams {
  uint64_t seed;
  uint64_t sweep;       // Philox sweep counter of this sweep
  int measure, meas_first, meas_last;
  int n_chains;
};

// launchers (dqmc_su2.cu)
size_t su2_smem_bytes(int maxN, int maxMV);
cudaError_t su2_launch_init_fields(Su2Dev* chains, int n_chains, uint64_t seed, cudaStream_t st);
// mode 0: recompute the left chain and G(0) of every chain, write the working
// G, log|det|, arg and the phase P; mode 1: the same for chain `only` into
// `out` ([N][N] complex) without touching the working G or P
cudaError_t su2_launch_fresh(Su2Dev* chains, int n_chains, int mode, int only, double2* out, size_t smem,
                             cudaStream_t st);
cudaError_t su2_launch_sweep(Su2Dev* chains, const Su2SweepParams& p, size_t smem, cudaStream_t st);
cudaError_t su2_launch_copy_green(Su2Dev* chains, int chain, double2* out, cudaStream_t st);
cudaError_t su2_launch_reset_stats(Su2Dev* chains, int n_chains, int clear_meas, cudaStream_t st);
// time-displaced measurement of every chain (only < 0) or of chain `only` (with
// its G(n_tau,0), G(0,n_tau) into gt0 / g0t): out_a [n_chains][n_tau+1] complex
// traces of G(tau,0), out_prec [n_chains][2] (mean, max) of Precision tau
cudaError_t su2_launch_tau(Su2Dev* chains, int n_chains, int only, int n_tau, double2* out_a, double* out_prec,
                           double2* gt0, double2* g0t, size_t smem, cudaStream_t st);
// per chain: CSR lists of the pair classes (off[c], pairs[c]: device pointers),
// ncls [n_chains]; out [n_chains][max_cls][4] complex
cudaError_t su2_launch_corr(const Su2Dev* chains, int n_chains, const int* const* off, const int* const* pairs,
                            const int* ncls, int max_cls, double2* out, cudaStream_t st);

}  // namespace dqmc
