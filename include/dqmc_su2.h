/* C ABI of the GB300 DQMC library: Markov chains of the SU(2)-symmetric
 * Hubbard model in the charge decoupling with complex coupling (the paper's
 * default Hubbard example, Sec. 6.1; discrete HS transform of Sec. 2.1;
 * complex weights and the phase of Sec. 2.2).
 *
 * Model.  H = sum_xy K_xy sum_s c+_xs c_ys + U/2 sum_i (n_i - 1)^2 with
 * n_i = n_i,up + n_i,dn.  The four-valued transform of Sec. 2.1 applied to
 * exp(-dtau U/2 (n_i - 1)^2) has an imaginary coupling:
 *   exp(-dtau U/2 (n_i - 1)^2) = sum_l gamma(l)/4 exp(i g eta(l) (n_i - 1)) + O(dtau^4),
 *   g = sqrt(dtau U / 2),  l in {-2, -1, 1, 2}.
 * Both colors see the same propagator B_tau = exp(-dtau K) exp(V_tau),
 * V_tau = diag(i g eta(l_tau,x)), so one complex N x N Green function
 * G(tau) = (1 + B(tau,0) B(beta,tau))^-1 serves both, and the weight is
 *   prod gamma(l)/4 * exp(-i g sum eta(l)) * det(1 + B(beta,0))^2.
 * Sampling uses W = |Re e^{-S}| (Sec. 2.2) with the phase
 * P = e^{-S}/|e^{-S}| = exp(i (-g sum eta + 2 arg det(1 + B(beta,0)))) carried
 * through the updates; observables are reweighted by sign * P / Re P.
 *
 * Bond model (optional, n_bonds > 0): the Hubbard-Ising model of Sec. 6, the
 * hopping on bond b = (i, j) coupled to an Ising spin s_b = +-1 with a
 * transverse field h and a coupling J between paired bonds.  Per slice the
 * two-site type-1 factors X_b = exp(-dtau xi s_b (|i><j| + |j><i|)) enter
 * B_tau = exp(-dtau K) X_0 X_1 ... X_{nb-1} exp(V_tau), and the weight gains
 * the spins' own factor prod_{tau,b} [cosh(dtau h) if s_b(tau) = s_b(tau+1)
 * else sinh(dtau h)] * exp(dtau J sum_{tau, pairs} s_b s_b') (periodic in tau).
 * Within a slice the vertices are visited in the order their factors act:
 * up the sites 0..N-1, then the bonds nb-1..0; down the reverse.  A bond
 * proposal is the flip s -> -s with the ratio det(1 + delta (1 - G~)_PP)^2
 * times the spins' weight ratio, and a rank-2 (Woodbury) update of G~; its
 * acceptance uniform comes from the Philox counter of vertex N + b.
 *
 * Arithmetic: complex FP64 throughout (G, wraps, rank-1 updates, the complex
 * pivoted-QR UDV chain and the stable G of Sec. 2.3).  One CTA per chain.
 *
 * Sweep order and random numbers as dqmc.h: up tau = 1..L with sites 0..N-1,
 * down tau = L..1 with sites N-1..0; Philox4x32-10 with key
 * (seed_lo, seed_hi ^ chain) and counter (sweep_lo, 2 tau + dir, site,
 * sweep_hi); u1 from words 0, 1 picks one of the three other field values
 * (ascending, index floor(3 u1)), u2 from words 2, 3 is the acceptance
 * uniform.  The sweep counter of a context starts at 0.
 *
 * Errors: dqmc_status codes of dqmc.h, no exceptions, no device traps.  A
 * context is used from one host thread at a time.
 */
#ifndef DQMC_SU2_H
#define DQMC_SU2_H

#include <stdint.h>

#include "dqmc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dqmc_su2_ctx dqmc_su2_ctx; /* opaque, library-owned */

typedef struct {
  int32_t n_sites;        /* N, 1..1024                                           */
  const double* hopping;  /* K [N][N] row-major, symmetric, -mu on the diagonal  */
  double U;               /* Hubbard U >= 0 (g = sqrt(dtau U / 2))               */
  double dtau;            /* > 0                                                  */
  int32_t L;              /* Trotter slices >= 1                                  */
  int32_t n_wrap;         /* stabilisation interval; L % n_wrap == 0 (Sec. 2.3)   */
  int32_t n_bonds;        /* Ising spins on bonds; 0: the plain SU(2) model       */
  const int32_t* bond_sites; /* [n_bonds][2] sites (i, j), i != j, in [0, N)       */
  double xi;              /* coupling of s_b to the hopping of its bond           */
  double h;               /* transverse field of the bond spins, > 0 with bonds   */
  double J;               /* coupling of paired bond spins                        */
  int32_t n_pairs;        /* J pairs                                              */
  const int32_t* pairs;   /* [n_pairs][2] bonds (b, b'), b != b', in [0, n_bonds) */
} dqmc_su2_model_desc;

typedef struct {
  int32_t measure;            /* nonzero: accumulate the energy estimator        */
  int32_t meas_first;         /* measure G(tau) for meas_first <= tau <= meas_last*/
  int32_t meas_last;          /*   (upward tau = 1..L, downward tau-1 = L-1..0)   */
  uint64_t seed;              /* Philox key (seed_lo, seed_hi ^ chain)            */
  double unstable_threshold;  /* > 0: DQMC_EUNSTABLE when prec_green_max or
                                 prec_phase_max exceeds it                       */
} dqmc_su2_opts;

typedef struct {
  int64_t proposals, accepted;
  double prec_green_mean;     /* "Precision Green" over the stabilisation events: */
  double prec_green_max;      /*   mean of mean |G_wrap - G_fresh|, max of max    */
  double prec_phase_max;      /* "Precision Phase": max |P_carried - P_fresh|     */
  double mean_sign;           /* mean over chains and sweeps of sign(Re P)        */
  float ms_total;             /* device time of the call (CUDA events)            */
} dqmc_su2_sweep_stats;

/* Create a context with n_chains chains; chain c uses models[chain_model[c]].
 * fields_or_null: packed per chain [L_c][N_c + n_bonds_c] (int8, host): per
 * slice the site fields in {-2,-1,1,2}, then the bond spins in {-1,1}; NULL
 * draws them i.i.d. uniform from Philox (counter (0xFFFFFFFF, tau, vertex,
 * 0xFFFFFFFF), vertex x for site x and N + b for bond b).  The left chain,
 * G(0), log|det|, arg det and the phase P are computed before return.  Inputs
 * are copied.
 * Errors: DQMC_EINVAL (bad model, options or field values), DQMC_ENOMEM,
 * DQMC_ECUDA, DQMC_EUNSTABLE (a singular matrix in the stabilisation).  On an
 * error *out may still receive a context that only carries the message. */
dqmc_status dqmc_su2_init(const dqmc_su2_model_desc* models, int32_t n_models, const int32_t* chain_model,
                          int32_t n_chains, const int8_t* fields_or_null, const dqmc_su2_opts* opts,
                          void* cuda_stream, dqmc_su2_ctx** out);

/* n_sweeps >= 1 sweeps of every chain (Algorithm 1); stats_or_null receives
 * the statistics of the call.  Blocks until the sweeps are done.
 * DQMC_EUNSTABLE: a singular matrix, or a precision figure above the
 * threshold (the sweeps still ran). */
dqmc_status dqmc_su2_sweep(dqmc_su2_ctx* ctx, int32_t n_sweeps, dqmc_su2_sweep_stats* stats_or_null);

/* G(0) of one chain ([N][N] complex, re/im interleaved, row-major) into out
 * (host, or device when out_is_device): fresh = 0 the working G the sweeps
 * left, fresh = 1 recomputed from the fields through the UDV chain.
 * logabs_out / arg_out (nullable): log|det(1 + B(beta,0))| and its argument
 * at the last fresh G; phase_out (nullable, [2]): the chain's phase P.
 * Errors: DQMC_ESTATE (no context), DQMC_EINVAL (chain out of range, null out),
 * DQMC_ECUDA, DQMC_EUNSTABLE (fresh = 1 met a singular matrix). */
dqmc_status dqmc_su2_greens(dqmc_su2_ctx* ctx, int32_t chain, int32_t fresh, double* out, int32_t out_is_device,
                            double* logabs_out, double* arg_out, double* phase_out);

/* Reweighted sums since the context was created or last measured-and-reset
 * (reset = 1): out [n_chains][5][2] = (re, im) of sum sign * P / Re P * O for
 * O = Kin, Pot, Part, Ener (Sec. 6.1 estimator, both colors; Kin of the hopping
 * K alone) and the bond spins' (sum_b s_b)^2 / n_bonds averaged over the slices
 * (0 without bonds); sign_sum [n_chains] = sum of sign(Re P); n_meas
 * [n_chains].  Host buffers, each nullable (skipped).  Waits for the context's
 * stream.  Errors: DQMC_ESTATE, DQMC_ECUDA. */
dqmc_status dqmc_su2_measure(dqmc_su2_ctx* ctx, double* out, double* sign_sum, int64_t* n_meas, int32_t reset);

/* Time-displaced measurement of every chain's current configuration (the tau_m
 * step, Sec. 2.4; the time-displaced observables of Sec. 5.2): from the stable
 * G(0), G(tau,0) = B_tau G(tau-1,0) and G(0,tau) = G(0,tau-1) B_tau^-1 for
 * tau = 1..n_tau, both recomputed from the UDV chains at every multiple of
 * n_wrap (G(tau,0) = (B(tau,0)^-1 + B(beta,tau))^-1, G(0,tau) =
 * -(1 - G(0)) B(tau,0)^-1).  out (host) [n_chains][n_tau + 1][2]: (re, im) of
 * sum_x G(tau,0)_xx; prec_tau (host, nullable) [2]: "Precision tau", the mean
 * over chains and recompute points of the mean |wrapped - recomputed| entry
 * of G(tau,0) and G(0,tau), and the maximum.  0 <= n_tau <= L of every chain.
 * The chains are left as they are.  Errors: DQMC_ESTATE, DQMC_EINVAL (null out,
 * n_tau out of range), DQMC_ENOMEM, DQMC_ECUDA, DQMC_EUNSTABLE (a singular
 * matrix at a recompute point). */
dqmc_status dqmc_su2_measure_tau(dqmc_su2_ctx* ctx, int32_t n_tau, double* out, double* prec_tau);

/* G(tau,0) and G(0,tau) of one chain ([N][N] complex each, host), reached as
 * dqmc_su2_measure_tau reaches them (wrapped from the last recompute point at
 * or below tau).  Errors: DQMC_ESTATE, DQMC_EINVAL (chain or tau out of range,
 * a null output), DQMC_ENOMEM, DQMC_ECUDA, DQMC_EUNSTABLE. */
dqmc_status dqmc_su2_greens_displaced(dqmc_su2_ctx* ctx, int32_t chain, int32_t tau, double* out_t0, double* out_0t);

/* Equal-time correlation functions of every chain's current configuration from
 * its working G(0) (the paper's SpinZ, Den, SpinXY and Green observables of
 * Sec. 6, collected per class of site pairs as Obser_Latt collects them per
 * displacement).  Both colors share G; with X_xy = (delta_xy - G_yx) G_xy and
 * rho_x = 2 (1 - G_xx), per configuration
 *     <S^z_x S^z_y> = X_xy / 2,  <n_x n_y> = rho_x rho_y + 2 X_xy,
 *     <S^+_x S^-_y> = X_xy,      sum_s <c^+_xs c_ys> = 2 (delta_xy - G_yx).
 *     pair_class  host, per model [n_sites][n_sites] int32 (models concatenated):
 *                 class of (x, y) in [0, n_class[m]), or -1 to skip it
 *     n_class     host [n_models], each >= 1
 * Outputs (host): out [n_chains][max n_class][4][2]: (re, im) of the sums over
 * each class's pairs (unweighted; rows beyond the chain's model's n_class are
 * 0); phase [n_chains][2]: the chain's phase P (reweight by sign(Re P) P / Re P).
 * The chains are left as they are.  DQMC_EINVAL for a class out of range. */
dqmc_status dqmc_su2_measure_corr(dqmc_su2_ctx* ctx, const int32_t* pair_class, const int32_t* n_class, double* out,
                                  double* phase);

/* Fields of every chain (packed [L_c][N_c + n_bonds_c] int8, host; out nullable)
 * and the sweep counter (nullable).  Errors: DQMC_ESTATE, DQMC_ECUDA. */
dqmc_status dqmc_su2_get_fields(dqmc_su2_ctx* ctx, int8_t* out, uint64_t* sweep_counter);
/* Replace the fields (host, packed as dqmc_su2_get_fields writes them) and the
 * sweep counter; the left chains, G(0) and the phases are recomputed.  Every
 * value is checked first; an invalid one returns DQMC_EINVAL and changes
 * nothing.  Errors: DQMC_ESTATE, DQMC_EINVAL, DQMC_ECUDA, DQMC_EUNSTABLE. */
dqmc_status dqmc_su2_set_fields(dqmc_su2_ctx* ctx, const int8_t* in, uint64_t sweep_counter);

const char* dqmc_su2_last_error(const dqmc_su2_ctx* ctx);
void dqmc_su2_destroy(dqmc_su2_ctx* ctx); /* NULL-safe */

#ifdef __cplusplus
}
#endif

#endif /* DQMC_SU2_H */
