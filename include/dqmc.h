/*
 * dqmc.h -- C ABI of the GB300 (sm_103a) library for the finite-temperature
 * auxiliary-field (BSS / DQMC) sweep documented in the ALF 1.0 paper
 * (Assaad et al., arXiv:1704.00131).
 *
 * The library runs Markov chains of Hubbard-type models on one GPU.  For a
 * field configuration C the weight is prod_s det(1 + B^s(beta,0)) (Sec. 2.1,
 * Eq. partition_2), with the one-slice propagator
 *     B^s_tau = exp(-dtau K^s) exp(V^s_tau),   V^s_tau = diag(v^s_i,tau),
 *     v^s_i,tau = sigma^s_k c(field_k,tau)  at site i = vertex_site[k],
 * and the equal-time Green function G^s(tau) = (1 + B^s(tau,0) B^s(beta,tau))^-1
 * (Eq. Green_eq).  Field types:
 *     DQMC_FIELD_ISING (paper type 1): fields +-1, c(s) = lambda s with
 *         cosh(lambda) = exp(dtau U / 2): the exact two-valued decoupling of
 *         exp(-dtau U (n_up - 1/2)(n_dn - 1/2)) for sigma = (+1, -1);
 *     DQMC_FIELD_HS4 (paper type 2, Sec. 2.1): fields -2,-1,1,2,
 *         c(l) = sqrt(dtau U / 2) eta(l) with weights gamma(l) (M_z Hubbard,
 *         Sec. 6.2).
 * A sweep visits every field twice, tau = 1..L then L..1 (Sec. 2.4,
 * Algorithm 1), proposes single-field changes accepted with
 * min(1, |W'/W|) (Sec. 2.2.1), wraps G between slices and recomputes it
 * from a QR-stabilised UDV chain every n_wrap slices (Sec. 2.3).
 *
 * Conventions for every entry point:
 *   - Matrices are row-major, dense, double precision on the host unless the
 *     argument says otherwise.
 *   - The library owns the context and every device buffer; inputs are copied
 *     at the call.  Outputs go to caller buffers.
 *   - Work is enqueued on the CUDA stream given at dqmc_init; a call that
 *     returns host data synchronises that stream before returning.
 *   - Errors are reported by the returned status only (no exceptions, no
 *     abort, no device trap); dqmc_last_error(ctx) gives a message.
 *   - One context per host thread.
 *   - No CPU fallback: every step of the sweep runs in the library's CUDA
 *     kernels; without a usable GPU dqmc_init returns DQMC_ECUDA.
 */
#ifndef DQMC_H_
#define DQMC_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dqmc_ctx dqmc_ctx; /* opaque, library-owned */

typedef enum {
  DQMC_OK = 0,
  DQMC_EINVAL = 1,    /* an argument is out of range or inconsistent          */
  DQMC_ENOMEM = 2,    /* device or host allocation failed                      */
  DQMC_ECUDA = 3,     /* a CUDA call failed (message in dqmc_last_error)       */
  DQMC_EUNSTABLE = 4, /* stabilisation failed, or max|G_wrap - G_fresh|
                         exceeded dqmc_run_opts.unstable_threshold             */
  DQMC_ETIMEOUT = 5,  /* a bounded device wait gave up (the tensor-core products
                         of DQMC_PREC_MIXED_TC wait on their copies and MMAs) */
  DQMC_ESTATE = 6     /* the call is not valid in the context's state          */
} dqmc_status;

typedef enum { DQMC_FIELD_ISING = 1, DQMC_FIELD_HS4 = 2 } dqmc_field_type;

/* Arithmetic of each precision mode.  The scales D of the UDV chains (which
 * reach e^100 and more) are FP64 in every mode.
 *   DQMC_PREC_FP64: everything in FP64: working G, wraps, delayed updates, the
 *     B-chain products, the pivoted QR, the T update, (1 + UDV)^-1 and log|det|
 *     (Sec. 2.3).
 *   DQMC_PREC_FP32: working G, wraps and delayed updates in plain FP32; the
 *     stabilisation in FP64 as above.  Round-off grows by the condition number of
 *     the unstabilised slice product (Sec. 2.3), so at strong coupling the wrapped
 *     G drifts far from the fresh one; the precision monitor reports it.
 *   DQMC_PREC_MIXED: float pairs (hi + lo, about 48 significant bits, error-free
 *     transformations on the FP32 pipes) for the working G, the wraps and the
 *     delayed updates, and also for the stabilisation: the B-chain and T-update
 *     products, the Householder QR (pivot chosen in FP64 on the FP64-scaled column
 *     norms), Q^T Q, T T^T, the LU of the middle matrix and the solves, with the
 *     FP64 scales D kept apart.  This departs from an FP64 stabilisation: the
 *     float-pair products accumulate about 42 bits, and the stable G then differs
 *     from an FP64 recompute by up to ~30x the FP64 round-off amplified by the
 *     conditioning (measured: 1e-9 at U = 4 - 6, beta = 4 - 8, n_wrap = 10 on
 *     equilibrated fields; up to 2e-6 on i.i.d. fields at U = 6, beta = 8, where
 *     FP64 itself moves by 3e-8 between n_wrap = 10 and 5).  The wrapped G between
 *     stabilisations drifts ~25x further than on the FP64 path (monitor).
 *   DQMC_PREC_MIXED_TC: as DQMC_PREC_MIXED, with every N x N x N product (wraps,
 *     B chain, T update, Q^T Q, T T^T, Q Y) an exact-split BF16 product on the
 *     tensor cores (tcgen05: seven 8-bit digits per operand, digit diagonals
 *     accumulated exactly in FP32 tensor memory, recombined in float pairs, about
 *     55 bits), so the products are as accurate as FP64 ones; QR, LU and solves
 *     stay float pairs.  Needs device memory for the digit planes and half of the
 *     tensor memory of each SM while a sweep runs. */
typedef enum {
  DQMC_PREC_FP64 = 0,
  DQMC_PREC_FP32 = 1,
  DQMC_PREC_MIXED = 2,
  DQMC_PREC_MIXED_TC = 3
} dqmc_precision;

/* One model: a lattice with its couplings (Sec. 3.1, the Operator type with
 * hopping Op_T, g = -dtau, and single-site vertices Op_V).  Chains refer to a
 * model by index; every model of one context has the same n_flavors. */
typedef struct {
  int32_t n_sites;            /* N >= 1                                            */
  int32_t n_flavors;          /* 1 or 2 (2 = spin up, spin down)                   */
  const double* hopping;      /* [n_flavors][N][N], symmetric, -mu on the diagonal */
  int32_t n_vertices;         /* M_V, 1 <= M_V <= N                                */
  const int32_t* vertex_site; /* [M_V] distinct sites in [0, N)                    */
  const double* vertex_sign;  /* [n_flavors][M_V] sigma^s_k (+1 / -1 for M_z)      */
  double U;                   /* >= 0                                              */
  int32_t field_type;         /* dqmc_field_type                                   */
  double dtau;                /* > 0; beta = L dtau                                */
  int32_t L;                  /* Trotter slices >= 1                               */
  int32_t n_wrap;             /* stabilisation interval; L % n_wrap == 0 (Sec. 2.3)*/
} dqmc_model_desc;

typedef struct {
  int32_t precision;          /* dqmc_precision                                    */
  int32_t delay_k;            /* accepted flips per delayed rank-k flush, 1..64    */
  int32_t measure;            /* nonzero: accumulate the energy estimator          */
  int32_t meas_first;         /* measure G(tau) for meas_first <= tau <= meas_last */
  int32_t meas_last;          /*   (upward tau = 1..L, downward tau-1 = L-1..0)    */
  uint64_t seed;              /* Philox key (seed_lo, seed_hi ^ chain)             */
  double unstable_threshold;  /* > 0: DQMC_EUNSTABLE when prec_green_max exceeds it*/
  int64_t spin_limit;         /* SM cycles before a bounded device wait gives up
                                 (DQMC_ETIMEOUT); 0: about one second            */
  int32_t tc_min_sites;       /* DQMC_PREC_MIXED_TC: chains of fewer sites use the
                                 float-pair SIMT products (0: 96, where the tensor-
                                 core product overtakes them on GB300)            */
  int32_t dd_tile;            /* float-pair SIMT products: output tiles of 48 x 48
                                 (3) or 64 x 64 (4) per CTA; 0: the one that pads
                                 the matrix least                                 */
  int32_t test_stall;         /* test hook, 0 in production: nonzero makes the
                                 first bounded wait of every tensor-core product
                                 wait on a barrier that nothing arrives on, so it
                                 gives up after spin_limit cycles; the call then
                                 reports DQMC_ETIMEOUT with the context usable    */
  int32_t stab_svd;           /* decomposition of the stabilisation chain: 0 the
                                 pivoted QR (default), 1 one-sided Jacobi SVD,
                                 Q = U, D = S, T = V^T T (the SVD alternative of
                                 Sec. 2.3 / the -DSTAB1 build option of Sec. 5);
                                 DQMC_PREC_FP64 only, DQMC_EINVAL otherwise     */
} dqmc_run_opts;

/* Statistics of one dqmc_sweep call, over all chains (Sec. 4.5 "info" file:
 * "Precision Green" mean and max, "Precision Phase", acceptance). */
typedef struct {
  int64_t proposals;          /* 2 L M_V per chain per sweep                       */
  int64_t accepted;
  double prec_green_mean;     /* mean over events of mean_ij |G_wrap - G_fresh|    */
  double prec_green_max;      /* max over events of max_ij |G_wrap - G_fresh|      */
  double prec_phase_max;      /* max |sign_tracked - sign_fresh|                   */
  double mean_sign;           /* mean over chains and sweeps of the end-of-sweep sign */
  float ms_total;             /* device time of the call (CUDA events)             */
  float ms_update;            /* the slowest chain's time in the updates (a4, a5), */
  float ms_wrap;              /*   the wraps (a3, a6), the stabilisation (a7-a10)  */
  float ms_stab;              /*   and the measurement (a12), from SM cycle        */
  float ms_measure;           /*   counters at the device's clock rate             */
  float ms_detail[8];         /* the same chain: ratio precompute, acceptance scan,
                                 update vectors, flushes, B-chain products, QR and
                                 Q, T update, stable G                             */
} dqmc_sweep_stats;

/* Create a context with n_chains chains; chain c uses models[chain_model[c]].
 * fields_or_null: packed per chain [L_c][M_V_c] (int8, host); NULL draws them
 * i.i.d. from Philox (counter (0xFFFFFFFF, tau, k, 0xFFFFFFFF)).  The initial
 * left chain and G(0) are computed before return (Algorithm 1, first loop).
 * cuda_stream: a cudaStream_t, or NULL for the default stream.
 * Errors: DQMC_EINVAL (bad model or options), DQMC_ENOMEM, DQMC_ECUDA,
 * DQMC_EUNSTABLE (the initial stabilisation hit a singular matrix).  On an
 * error *out may still receive a context that only carries the message for
 * dqmc_last_error; the caller destroys it with dqmc_destroy. */
dqmc_status dqmc_init(const dqmc_model_desc* models, int32_t n_models, const int32_t* chain_model,
                      int32_t n_chains, const int8_t* fields_or_null, const dqmc_run_opts* opts,
                      void* cuda_stream, dqmc_ctx** out);

/* Run n_sweeps sweeps of every chain (Algorithm 1).  With stats_or_null == NULL
 * the call only enqueues work and returns immediately; otherwise it waits for
 * the sweeps and fills *stats_or_null.  Errors: DQMC_EINVAL (n_sweeps < 0),
 * DQMC_ECUDA, DQMC_EUNSTABLE. */
dqmc_status dqmc_sweep(dqmc_ctx* ctx, int32_t n_sweeps, dqmc_sweep_stats* stats_or_null);

/* Equal-time Green function G^flavor(0) of one chain between sweeps (Eq.
 * Green_eq).  fresh = 0: the library's working G (FP64, or the FP32 / float-pair
 * values of the reduced-precision modes widened to FP64); fresh = 1: recomputed
 * from the fields through the FP64 UDV chain (Sec. 2.3).  out: N x N doubles, host (out_is_device = 0) or device.
 * logdet_out / sign_out (nullable): log|det(1 + B(beta,0))| and its sign from
 * the last stable recompute of that flavor. */
dqmc_status dqmc_greens(dqmc_ctx* ctx, int32_t chain, int32_t flavor, int32_t fresh, double* out,
                        int32_t out_is_device, double* logdet_out, int32_t* sign_out);

/* Equal-time Green function G^flavor(tau) of one chain on its current fields,
 * wrapped in the context's working precision the way the upward pass of a sweep
 * carries it between stabilisations when no proposal is accepted (Sec. 2.3, the
 * wrapped Green function whose drift the "Precision Green" monitor measures;
 * Algorithm 1, wrapgrup): the stable G(tau0) at the last stabilisation point
 * tau0 = n_wrap floor(tau / n_wrap), from the right chain B(tau0,0) and the
 * stored left chain B(beta,tau0)^T in the working precision's stabilisation
 * arithmetic, followed by tau - tau0 wraps G <- B_t G B_t^-1.  Call it between
 * sweeps (the stored chain then holds the left chain).  tau in [0, L]; out: N x N
 * doubles, host (out_is_device = 0) or device.  The chain's fields, working G
 * and stored chain are left as they are.  Errors: DQMC_EINVAL, DQMC_ECUDA,
 * DQMC_EUNSTABLE (singular middle matrix). */
dqmc_status dqmc_greens_tau(dqmc_ctx* ctx, int32_t chain, int32_t flavor, int32_t tau, double* out,
                            int32_t out_is_device);

/* Sign-weighted sums of the energy estimator since dqmc_init (Sec. 6.1
 * observables in the U n_up n_dn form):
 *     out[c][0] = sum sign * Kin,  Kin  = sum_s sum_xy K^s_xy (delta_xy - G^s_yx)
 *     out[c][1] = sum sign * Pot,  Pot  = U sum_i (1 - G^up_ii)(1 - G^dn_ii)
 *     out[c][2] = sum sign * Part, Part = sum_s sum_i (1 - G^s_ii)
 *     out[c][3] = sum sign * (Kin + Pot)
 * sign_sum[c] = sum of signs, n_meas[c] = number of measurements (host arrays).
 * Waits for the context's stream.  Errors: DQMC_EINVAL (a null output),
 * DQMC_ECUDA. */
dqmc_status dqmc_measure(dqmc_ctx* ctx, double* out, double* sign_sum, int64_t* n_meas);

/* Time-displaced Green functions of every chain's current configuration: the
 * tau measurement at the end of a sweep (Algorithm 1), giving the quantities
 * that ObserT receives (Sec. 5.2), with the "Precision tau" monitor of the
 * wrapped against the recomputed time-displaced functions (Sec. 2.3, info file).
 * From G(0) the library wraps, slice by slice,
 *     G(tau,0) = B_tau G(tau-1,0),   G(0,tau) = G(0,tau-1) B_tau^-1,
 *     G(tau,tau) = B_tau G(tau-1,tau-1) B_tau^-1,
 * with G(0,0) = G(0), G(0,0^+) = -(1 - G(0)), and replaces all three by the
 * stable recompute from the UDV chains at every tau = j n_wrap (FP64 throughout,
 * whatever the sweep precision).  The fields, the working G and the stored
 * chains of the ensemble are left as they are.
 *     n_tau      chain c measures tau = 0 .. min(n_tau, L_c); 0 <= n_tau <= max L
 *     site_phase host [sum over models of n_sites] (model order) phases ph_x,
 *                or NULL for ph = 1
 * Outputs (host):
 *     out  [n_chains][n_tau + 1][n_flavors][3]:
 *            a = sum_x G^s(tau,0)_xx,
 *            c = -sum_xy ph_x ph_y G^s(0,tau)_yx G^s(tau,0)_xy,
 *            p = sum_x ph_x (1 - G^s(tau,tau)_xx);  rows tau > L_c are 0.
 *          For the spin-z decoupling (flavor 0 up, 1 down),
 *            sum_xy ph_x ph_y <S^z_x(tau) S^z_y(0)> =
 *              [(p_0(tau) - p_1(tau)) (p_0(0) - p_1(0)) + c_0(tau) + c_1(tau)] / 4
 *          and the local Green function is (a_0 + a_1) / (n_flavors N).
 *     sign [n_chains][n_flavors]: sign of det(1 + B^s(beta,0)) (multiply the
 *          flavors for the configuration's sign)
 *     prec [2] or NULL: mean over stabilisation points (chains, flavors) of the
 *          element-mean |wrapped - recomputed| of G(tau,0) and G(0,tau), and the
 *          largest element difference.
 * DQMC_EUNSTABLE if a recompute meets a singular matrix. */
dqmc_status dqmc_measure_tau(dqmc_ctx* ctx, int32_t n_tau, const double* site_phase, double* out, int32_t* sign,
                             double* prec);

/* Time-displaced correlation functions of every chain's current configuration
 * per class of site pairs: the lattice-resolved quantities that ObserT collects
 * (Sec. 5.2; Algorithm 1, the tau measurement at the end of a sweep), for the two
 * flavors of the spin-z decoupling (flavor 0 up, flavor 1 down; two-flavor
 * models only).  G^s(tau,0), G^s(0,tau) and G^s(tau,tau) are wrapped and
 * re-stabilised exactly as in dqmc_measure_tau (FP64), and with
 * n^s_x(tau) = 1 - G^s(tau,tau)_xx and X^s_xy = -G^s(0,tau)_yx G^s(tau,0)_xy
 * Wick's theorem per configuration gives
 *     sum_s <c_xs(tau) c^+_ys(0)> = sum_s G^s(tau,0)_xy
 *     <S^z_x(tau) S^z_y(0)> = [(n^0_x(tau) - n^1_x(tau)) (n^0_y(0) - n^1_y(0)) + X^0_xy + X^1_xy] / 4
 *     <n_x(tau) n_y(0)>     = (n^0_x(tau) + n^1_x(tau)) (n^0_y(0) + n^1_y(0)) + X^0_xy + X^1_xy
 *     n_tau       chain c measures tau = 0 .. min(n_tau, L_c); 0 <= n_tau <= max L
 *     pair_class  host, per model [n_sites][n_sites] int32 (models concatenated):
 *                 class of the pair (x, y) in [0, n_class[m]), or -1 to skip it
 *     n_class     host [n_models], each >= 1
 * Outputs (host):
 *     out  [n_chains][n_tau + 1][max over models of n_class][3]: per class the
 *          sums over its pairs of the three expectation values above
 *          (unweighted); rows tau > L_c and classes beyond the chain's model's
 *          n_class are 0
 *     sign [n_chains]: sign of the configuration's weight (product of the
 *          flavors' det signs)
 * The chains are left as they are.  Errors: DQMC_EINVAL (one-flavor model, a
 * class outside [-1, n_class), n_tau out of range), DQMC_ENOMEM, DQMC_ECUDA,
 * DQMC_EUNSTABLE. */
dqmc_status dqmc_measure_tau_corr(dqmc_ctx* ctx, int32_t n_tau, const int32_t* pair_class, const int32_t* n_class,
                                  double* out, int32_t* sign);

/* Equal-time correlation functions of every chain's current configuration (the
 * equal-time observables of Sec. 5.2 and the correlation functions of Sec. 6,
 * collected per class of site pairs as Obser_Latt collects them per lattice
 * displacement), from the working G(0) of the two flavors of the spin-z
 * decoupling (flavor 0 up, flavor 1 down; two-flavor models only).  With
 * X^s_xy = (delta_xy - G^s_yx) G^s_xy, Wick's theorem per configuration gives
 *     <S^z_x S^z_y> = [m_x m_y + X^0_xy + X^1_xy] / 4,  m_x = G^1_xx - G^0_xx
 *     <n_x n_y>     = rho_x rho_y + X^0_xy + X^1_xy,    rho_x = 2 - G^0_xx - G^1_xx
 *     <S^+_x S^-_y> = (delta_xy - G^0_yx) G^1_xy
 *     sum_s <c^+_xs c_ys> = sum_s (delta_xy - G^s_yx)
 *     pair_class  host, per model [n_sites][n_sites] int32 (models concatenated):
 *                 class of the pair (x, y) in [0, n_class[m]), or -1 to skip it
 *     n_class     host [n_models], each >= 1
 * Outputs (host):
 *     out  [n_chains][max over models of n_class][4]: per class the sums over its
 *          pairs of the four expectation values above (unweighted; rows beyond
 *          the chain's model's n_class are 0)
 *     sign [n_chains]: sign of the configuration's weight (multiply before averaging)
 * The chains are left as they are.  DQMC_EINVAL for a one-flavor model or a
 * class outside [-1, n_class). */
dqmc_status dqmc_measure_corr(dqmc_ctx* ctx, const int32_t* pair_class, const int32_t* n_class, double* out,
                              int32_t* sign);

/* Derivatives of log|det(1 + B^s(beta,0))| on fixed field configurations of
 * model `model_index` (FP64):
 *     d log|det| = sum_tau Tr[(1 - G(tau-1)) B_tau^-1 dB_tau]
 * (from Eq. Green_eq by d log det(1 + B) = Tr[(1 + B)^-1 dB]).
 * fields: [n_cfg][L][M_V] int8 host.  Outputs (host):
 *     logdet  [n_cfg][n_flavors]
 *     grad_K  [n_cfg][n_flavors][N][N]: d/dK^s_xy with K_xy and K_yx varied
 *             together (x != y); d/dK_xx on the diagonal
 *     grad_U  [n_cfg][n_flavors]: d/dU through the couplings c(field).
 * The workspace (one FP64 chain per configuration) is allocated and freed by
 * the call, which waits for its work.  Errors: DQMC_EINVAL (model_index out of
 * range, n_cfg < 1, a null pointer, an invalid field value), DQMC_ENOMEM,
 * DQMC_ECUDA, DQMC_EUNSTABLE (a singular matrix in the stabilisation of a
 * configuration). */
dqmc_status dqmc_logdet_backward(dqmc_ctx* ctx, int32_t model_index, const int8_t* fields, int32_t n_cfg,
                                 double* logdet, double* grad_K, double* grad_U);

/* Derivatives of the energy estimator at tau = 0 (the Kin + Pot of dqmc_measure,
 * evaluated at G(0) = (1 + B(beta,0))^-1) on fixed field configurations of model
 * `model_index` (FP64).  With Gamma = dE/dG:
 *     dE = (explicit, at fixed G) + sum_s sum_tau Tr[G(tau-1,0) Gamma^T G(0,tau) dB_tau]
 * (dG = -G dB(beta,0) G with the time-displaced Green functions G(tau,0) =
 * B(tau,0) G(0) and G(0,tau) = -(1 - G(0)) B(tau,0)^-1, both computed stably
 * from the UDV chains).  fields: [n_cfg][L][M_V] int8 host.  Outputs (host):
 *     energy  [n_cfg][4] = Kin, Pot, Part, Ener of each configuration
 *     grad_K  [n_cfg][n_flavors][N][N]: dEner/dK^s_xy, K_xy and K_yx varied together
 *     grad_U  [n_cfg]: dEner/dU (explicit U and the couplings c(field)).
 * Workspace, waiting and errors as dqmc_logdet_backward. */
dqmc_status dqmc_energy_backward(dqmc_ctx* ctx, int32_t model_index, const int8_t* fields, int32_t n_cfg,
                                 double* energy, double* grad_K, double* grad_U);

/* Checkpoint: fields of every chain, packed [c][L_c][M_V_c] (host), and the
 * Philox sweep counter (confout / confin of Algorithm 1). */
dqmc_status dqmc_get_fields(dqmc_ctx* ctx, int8_t* out, uint64_t* rng_counter);
/* Resume: replaces the fields and the sweep counter and recomputes the left
 * chain and G(0) of every chain.  in: the packed fields as dqmc_get_fields
 * writes them.  Every value is checked first (+-1, or -2,-1,1,2 for
 * DQMC_FIELD_HS4); an invalid one returns DQMC_EINVAL and changes nothing. */
dqmc_status dqmc_set_fields(dqmc_ctx* ctx, const int8_t* in, uint64_t rng_counter);

/* Allocation-free computation of G^s(0) for every flavor (no counterpart in
 * the paper; it is a service of this library).  For callers that cannot
 * allocate device memory where they need G: code running under an allocator
 * that owns all device memory, or a context that must not call cudaMalloc.
 * It allocates nothing and needs no dqmc_ctx: all inputs and outputs are the
 * caller's device buffers, and its scratch is one device array of this library
 * (about 1 MiB, held by every GPU that loads the library until exit).
 *   Inputs (device): E_dev [n_flavors][N][N] = exp(-dtau K^s) row-major;
 *     vertex_site_dev [M_V]: distinct sites in [0, N) (the kernel checks this
 *     before it uses them; a violation gives sign 0, log|det| 0 and a G of
 *     NaNs); vertex_sign_dev [n_flavors][M_V]; fields_dev [L][M_V] int8 (+-1,
 *     or -2,-1,1,2 for DQMC_FIELD_HS4).
 *   Outputs (device): G_out_dev [n_flavors][N][N]; logdet_out_dev [n_flavors]
 *     and sign_out_dev [n_flavors] (nullable; sign 0 marks a singular
 *     stabilisation or invalid vertex sites).
 * Limits: N <= 64, n_flavors <= 2; larger sizes return DQMC_EINVAL before any
 * device work.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  The work is enqueued on cuda_stream (NULL: the
 * default stream) and the call returns without waiting.  Every call shares the
 * one array, so calls that overlap on the GPU (different streams, or different
 * host threads on the same device) race and give wrong results: serialise them.
 * Errors: DQMC_EINVAL, DQMC_ECUDA. */
dqmc_status dqmc_green_fresh_noalloc(int32_t n_sites, int32_t n_flavors, const double* E_dev, int32_t n_vertices,
                                     const int32_t* vertex_site_dev, const double* vertex_sign_dev, double U,
                                     int32_t field_type, double dtau, int32_t L, int32_t n_wrap,
                                     const int8_t* fields_dev, double* G_out_dev, double* logdet_out_dev,
                                     int32_t* sign_out_dev, void* cuda_stream);

/* Per-context message of the last failing call; valid until the next call. */
const char* dqmc_last_error(const dqmc_ctx* ctx);

/* Frees every resource of the context; NULL-safe. */
void dqmc_destroy(dqmc_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* DQMC_H_ */
