// Host side of the C ABI declared in include/dqmc_su2.h: validation, the
// exponentials exp(-+dtau K) of each model (Sec. 3.1, Op_set), the device arena
// of every chain of the SU(2) decoupling, and the launches of dqmc_su2.cu.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/dqmc_su2.h"
#include "dqmc_linalg_host.h"
#include "dqmc_su2_internal.h"

using dqmc::Su2Dev;

struct dqmc_su2_ctx {
  std::string err;
  cudaStream_t stream = nullptr;
  dqmc_su2_opts opts{};
  std::vector<dqmc_su2_model_desc> models;
  std::vector<int> chain_model;
  std::vector<Su2Dev> chains_h;
  Su2Dev* chains_d = nullptr;
  std::vector<void*> allocs;
  size_t smem = 0;
  uint64_t sweep_counter = 0;
  int maxN = 0, maxMV = 0;
  double2* out_scratch = nullptr;  // [maxN][maxN] complex for dqmc_su2_greens
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

namespace {

dqmc_status fail(dqmc_su2_ctx* ctx, dqmc_status st, const char* fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    ctx->err = buf;
  }
  return st;
}

#define SU2_CUDA_TRY(ctx, expr)                                                                  \
  do {                                                                                           \
    cudaError_t e_ = (expr);                                                                     \
    if (e_ != cudaSuccess) return fail((ctx), DQMC_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
  } while (0)

constexpr int kMaxSites = 1024;

dqmc_status validate(dqmc_su2_ctx* ctx, const dqmc_su2_model_desc& m, int idx) {
  if (m.n_sites < 1 || m.n_sites > kMaxSites)
    return fail(ctx, DQMC_EINVAL, "model %d: n_sites must be in 1..%d", idx, kMaxSites);
  if (!m.hopping) return fail(ctx, DQMC_EINVAL, "model %d: null hopping", idx);
  if (!(m.dtau > 0.0) || !std::isfinite(m.dtau)) return fail(ctx, DQMC_EINVAL, "model %d: dtau must be > 0", idx);
  if (!(m.U >= 0.0) || !std::isfinite(m.U)) return fail(ctx, DQMC_EINVAL, "model %d: U must be >= 0", idx);
  if (m.L < 1 || m.n_wrap < 1 || m.L % m.n_wrap != 0)
    return fail(ctx, DQMC_EINVAL, "model %d: need L >= 1, n_wrap >= 1 and L %% n_wrap == 0", idx);
  const int N = m.n_sites;
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) {
      const double a = m.hopping[(size_t)i * N + j], b = m.hopping[(size_t)j * N + i];
      if (!std::isfinite(a)) return fail(ctx, DQMC_EINVAL, "model %d: non-finite hopping", idx);
      if (std::fabs(a - b) > 1e-12 * (1.0 + std::fabs(a))) return fail(ctx, DQMC_EINVAL, "model %d: hopping not symmetric", idx);
    }
  if (m.n_bonds < 0 || m.n_pairs < 0) return fail(ctx, DQMC_EINVAL, "model %d: negative bond or pair count", idx);
  if (m.n_bonds > 0) {
    if (!m.bond_sites) return fail(ctx, DQMC_EINVAL, "model %d: null bond_sites", idx);
    if (!(m.h > 0.0) || !std::isfinite(m.h) || !std::isfinite(m.xi) || !std::isfinite(m.J))
      return fail(ctx, DQMC_EINVAL, "model %d: need a finite xi, J and h > 0 with bonds", idx);
    for (int b = 0; b < m.n_bonds; ++b) {
      const int i = m.bond_sites[2 * b], j = m.bond_sites[2 * b + 1];
      if (i < 0 || i >= N || j < 0 || j >= N || i == j)
        return fail(ctx, DQMC_EINVAL, "model %d: bond %d = (%d, %d) invalid", idx, b, i, j);
    }
  } else if (m.n_pairs > 0) {
    return fail(ctx, DQMC_EINVAL, "model %d: J pairs without bonds", idx);
  }
  if (m.n_pairs > 0 && !m.pairs) return fail(ctx, DQMC_EINVAL, "model %d: null pairs", idx);
  for (int q = 0; q < m.n_pairs; ++q) {
    const int a = m.pairs[2 * q], b = m.pairs[2 * q + 1];
    if (a < 0 || a >= m.n_bonds || b < 0 || b >= m.n_bonds || a == b)
      return fail(ctx, DQMC_EINVAL, "model %d: pair %d = (%d, %d) invalid", idx, q, a, b);
  }
  return DQMC_OK;
}

template <typename T>
dqmc_status dev_alloc(dqmc_su2_ctx* ctx, T** p, size_t n) {
  void* q = nullptr;
  if (cudaMalloc(&q, n * sizeof(T) + 16) != cudaSuccess) return fail(ctx, DQMC_ENOMEM, "cudaMalloc of %zu bytes", n * sizeof(T));
  ctx->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return DQMC_OK;
}

// fields of one chain, [L][N + nb]: sites in {-2, -1, 1, 2}, bond spins in {-1, 1}
dqmc_status check_fields(dqmc_su2_ctx* ctx, const int8_t* f, int L, int N, int MV) {
  for (int t = 0; t < L; ++t)
    for (int v = 0; v < MV; ++v) {
      const int x = f[(size_t)t * MV + v];
      const bool ok = (v < N) ? (x == 1 || x == -1 || x == 2 || x == -2) : (x == 1 || x == -1);
      if (!ok) return fail(ctx, DQMC_EINVAL, "field value %d at slice %d, vertex %d is invalid", x, t, v);
    }
  return DQMC_OK;
}

dqmc_status download(dqmc_su2_ctx* ctx) {
  SU2_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->chains_h.data(), ctx->chains_d, sizeof(Su2Dev) * ctx->chains_h.size(),
                                    cudaMemcpyDeviceToHost, ctx->stream));
  SU2_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return DQMC_OK;
}

// left chains, G(0), log|det|, arg and phase of every chain from its fields
dqmc_status refill(dqmc_su2_ctx* ctx) {
  const int n = (int)ctx->chains_h.size();
  SU2_CUDA_TRY(ctx, dqmc::su2_launch_reset_stats(ctx->chains_d, n, 0, ctx->stream));
  SU2_CUDA_TRY(ctx, dqmc::su2_launch_fresh(ctx->chains_d, n, 0, -1, nullptr, ctx->smem, ctx->stream));
  dqmc_status st = download(ctx);
  if (st) return st;
  for (const Su2Dev& C : ctx->chains_h)
    if (C.error) return fail(ctx, DQMC_EUNSTABLE, "chain %u: singular matrix in the stabilisation", C.chain_id);
  return DQMC_OK;
}

}  // namespace

extern "C" {

dqmc_status dqmc_su2_init(const dqmc_su2_model_desc* models, int32_t n_models, const int32_t* chain_model,
                          int32_t n_chains, const int8_t* fields, const dqmc_su2_opts* opts, void* cuda_stream,
                          dqmc_su2_ctx** out) {
  if (!out) return DQMC_EINVAL;
  *out = nullptr;
  dqmc_su2_ctx* ctx = new dqmc_su2_ctx();
  *out = ctx;
  if (!models || n_models < 1 || !chain_model || n_chains < 1 || !opts)
    return fail(ctx, DQMC_EINVAL, "null argument or empty model / chain list");
  ctx->opts = *opts;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  for (int i = 0; i < n_models; ++i) {
    dqmc_status st = validate(ctx, models[i], i);
    if (st) return st;
    ctx->models.push_back(models[i]);
  }
  for (int c = 0; c < n_chains; ++c) {
    if (chain_model[c] < 0 || chain_model[c] >= n_models)
      return fail(ctx, DQMC_EINVAL, "chain %d: model index %d out of range", c, chain_model[c]);
    ctx->chain_model.push_back(chain_model[c]);
  }
  if (opts->measure && opts->meas_first > opts->meas_last)
    return fail(ctx, DQMC_EINVAL, "meas_first > meas_last");
  SU2_CUDA_TRY(ctx, cudaEventCreate(&ctx->ev0));
  SU2_CUDA_TRY(ctx, cudaEventCreate(&ctx->ev1));
  // per model: K, E = exp(-dtau K), E^-1, the identity and a vector of ones, the
  // bonds and the CSR lists of the J pairs
  struct Dm { double *K, *E, *Einv, *ones; double2* ident; int ld; int *bi, *bj, *nbr_off, *nbr; };
  std::vector<Dm> dm(n_models);
  for (int i = 0; i < n_models; ++i) {
    const dqmc_su2_model_desc& m = models[i];
    const int N = m.n_sites, ld = N;
    std::vector<double> K(m.hopping, m.hopping + (size_t)N * N), w, V;
    dqmc::host::symmetric_eigen(N, K, w, V);
    const std::vector<double> E = dqmc::host::expm_symmetric(N, w, V, -m.dtau);
    const std::vector<double> Ei = dqmc::host::expm_symmetric(N, w, V, +m.dtau);
    for (double x : E)
      if (!std::isfinite(x)) return fail(ctx, DQMC_EINVAL, "model %d: exp(-dtau K) is not finite", i);
    for (double x : Ei)
      if (!std::isfinite(x)) return fail(ctx, DQMC_EINVAL, "model %d: exp(dtau K) is not finite", i);
    std::vector<double2> I((size_t)N * ld, make_double2(0.0, 0.0));
    for (int x = 0; x < N; ++x) I[(size_t)x * ld + x] = make_double2(1.0, 0.0);
    std::vector<double> ones(ld, 1.0);
    Dm& d = dm[i];
    d.ld = ld;
    dqmc_status st;
    if ((st = dev_alloc(ctx, &d.K, K.size())) || (st = dev_alloc(ctx, &d.E, E.size())) ||
        (st = dev_alloc(ctx, &d.Einv, Ei.size())) || (st = dev_alloc(ctx, &d.ident, I.size())) ||
        (st = dev_alloc(ctx, &d.ones, ones.size())))
      return st;
    SU2_CUDA_TRY(ctx, cudaMemcpy(d.K, K.data(), K.size() * sizeof(double), cudaMemcpyHostToDevice));
    SU2_CUDA_TRY(ctx, cudaMemcpy(d.E, E.data(), E.size() * sizeof(double), cudaMemcpyHostToDevice));
    SU2_CUDA_TRY(ctx, cudaMemcpy(d.Einv, Ei.data(), Ei.size() * sizeof(double), cudaMemcpyHostToDevice));
    SU2_CUDA_TRY(ctx, cudaMemcpy(d.ident, I.data(), I.size() * sizeof(double2), cudaMemcpyHostToDevice));
    SU2_CUDA_TRY(ctx, cudaMemcpy(d.ones, ones.data(), ones.size() * sizeof(double), cudaMemcpyHostToDevice));
    const int nb = m.n_bonds;
    std::vector<int> bi(nb + 1, 0), bj(nb + 1, 0), off(nb + 2, 0), nbr;
    for (int b = 0; b < nb; ++b) { bi[b] = m.bond_sites[2 * b]; bj[b] = m.bond_sites[2 * b + 1]; }
    std::vector<std::vector<int>> adj(nb);
    for (int q = 0; q < m.n_pairs; ++q) {
      adj[m.pairs[2 * q]].push_back(m.pairs[2 * q + 1]);
      adj[m.pairs[2 * q + 1]].push_back(m.pairs[2 * q]);
    }
    for (int b = 0; b < nb; ++b) {
      off[b + 1] = off[b] + (int)adj[b].size();
      nbr.insert(nbr.end(), adj[b].begin(), adj[b].end());
    }
    nbr.push_back(0);
    if ((st = dev_alloc(ctx, &d.bi, bi.size())) || (st = dev_alloc(ctx, &d.bj, bj.size())) ||
        (st = dev_alloc(ctx, &d.nbr_off, off.size())) || (st = dev_alloc(ctx, &d.nbr, nbr.size())))
      return st;
    SU2_CUDA_TRY(ctx, cudaMemcpy(d.bi, bi.data(), bi.size() * sizeof(int), cudaMemcpyHostToDevice));
    SU2_CUDA_TRY(ctx, cudaMemcpy(d.bj, bj.data(), bj.size() * sizeof(int), cudaMemcpyHostToDevice));
    SU2_CUDA_TRY(ctx, cudaMemcpy(d.nbr_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice));
    SU2_CUDA_TRY(ctx, cudaMemcpy(d.nbr, nbr.data(), nbr.size() * sizeof(int), cudaMemcpyHostToDevice));
    ctx->maxN = std::max(ctx->maxN, N);
    ctx->maxMV = std::max(ctx->maxMV, N + nb);
  }
  // per chain: one arena
  size_t foff = 0;
  for (int c = 0; c < n_chains; ++c) {
    const dqmc_su2_model_desc& m = models[chain_model[c]];
    const Dm& d = dm[chain_model[c]];
    const int N = m.n_sites, ld = d.ld, nst = m.L / m.n_wrap, MV = N + m.n_bonds;
    Su2Dev C{};
    C.N = N; C.ld = ld; C.L = m.L; C.nw = m.n_wrap;
    C.nb = m.n_bonds; C.MV = MV;
    C.dtau = m.dtau; C.U = m.U; C.g = std::sqrt(0.5 * m.dtau * m.U);
    C.a0 = -m.dtau * m.xi;
    if (m.n_bonds > 0) {
      C.lch = std::log(std::cosh(m.dtau * m.h));
      C.lsh = std::log(std::sinh(m.dtau * m.h));
      C.dJ = m.dtau * m.J;
    }
    C.bi = d.bi; C.bj = d.bj; C.nbr_off = d.nbr_off; C.nbr = d.nbr;
    C.K = d.K; C.E = d.E; C.Einv = d.Einv; C.ident = d.ident; C.ones = d.ones;
    C.chain_id = (uint32_t)c;
    dqmc_status st;
    if ((st = dev_alloc(ctx, &C.fields, (size_t)m.L * MV)) || (st = dev_alloc(ctx, &C.G, (size_t)N * ld)) ||
        (st = dev_alloc(ctx, &C.Gt, (size_t)N * ld)) ||
        (st = dev_alloc(ctx, &C.slots, (size_t)(nst + 1) * dqmc::su2_slot_elems(N, ld))) ||
        (st = dev_alloc(ctx, &C.slotD, (size_t)(nst + 1) * ld)) || (st = dev_alloc(ctx, &C.slot_detq, nst + 1)) ||
        (st = dev_alloc(ctx, &C.work, dqmc::su2_work_elems(N, ld))) ||
        (st = dev_alloc(ctx, &C.dwork, (size_t)dqmc::kSu2DVecs * ld)) || (st = dev_alloc(ctx, &C.iwork, ld)))
      return st;
    if (fields) {
      dqmc_status fs = check_fields(ctx, fields + foff, m.L, N, MV);
      if (fs) return fs;
      SU2_CUDA_TRY(ctx, cudaMemcpy(C.fields, fields + foff, (size_t)m.L * MV, cudaMemcpyHostToDevice));
    }
    foff += (size_t)m.L * MV;
    ctx->chains_h.push_back(C);
  }
  SU2_CUDA_TRY(ctx, cudaMalloc(&ctx->chains_d, sizeof(Su2Dev) * n_chains));
  SU2_CUDA_TRY(ctx, cudaMalloc(&ctx->out_scratch, sizeof(double2) * (size_t)ctx->maxN * ctx->maxN));
  SU2_CUDA_TRY(ctx, cudaMemcpy(ctx->chains_d, ctx->chains_h.data(), sizeof(Su2Dev) * n_chains,
                               cudaMemcpyHostToDevice));
  ctx->smem = dqmc::su2_smem_bytes(ctx->maxN, ctx->maxMV);
  if (!fields) SU2_CUDA_TRY(ctx, dqmc::su2_launch_init_fields(ctx->chains_d, n_chains, opts->seed, ctx->stream));
  SU2_CUDA_TRY(ctx, dqmc::su2_launch_reset_stats(ctx->chains_d, n_chains, 1, ctx->stream));
  return refill(ctx);
}

dqmc_status dqmc_su2_sweep(dqmc_su2_ctx* ctx, int32_t n_sweeps, dqmc_su2_sweep_stats* stats) {
  if (!ctx || !ctx->chains_d) return fail(ctx, DQMC_ESTATE, "context not initialised");
  if (n_sweeps < 1) return fail(ctx, DQMC_EINVAL, "n_sweeps must be >= 1");
  const int n = (int)ctx->chains_h.size();
  SU2_CUDA_TRY(ctx, dqmc::su2_launch_reset_stats(ctx->chains_d, n, 0, ctx->stream));
  SU2_CUDA_TRY(ctx, cudaEventRecord(ctx->ev0, ctx->stream));
  for (int s = 0; s < n_sweeps; ++s) {
    dqmc::Su2SweepParams p{};
    p.seed = ctx->opts.seed;
    p.sweep = ctx->sweep_counter++;
    p.measure = ctx->opts.measure;
    p.meas_first = ctx->opts.meas_first;
    p.meas_last = ctx->opts.meas_last;
    p.n_chains = n;
    SU2_CUDA_TRY(ctx, dqmc::su2_launch_sweep(ctx->chains_d, p, ctx->smem, ctx->stream));
  }
  SU2_CUDA_TRY(ctx, cudaEventRecord(ctx->ev1, ctx->stream));
  dqmc_status st = download(ctx);
  if (st) return st;
  float ms = 0.f;
  SU2_CUDA_TRY(ctx, cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
  dqmc_su2_sweep_stats S{};
  double prec_sum = 0.0, sign_sum = 0.0;
  int64_t events = 0;
  int err = 0;
  for (const Su2Dev& C : ctx->chains_h) {
    S.proposals += C.proposals;
    S.accepted += C.accepted;
    prec_sum += C.prec_sum;
    events += C.prec_events;
    S.prec_green_max = std::max(S.prec_green_max, C.prec_max);
    S.prec_phase_max = std::max(S.prec_phase_max, C.phase_max);
    sign_sum += C.sweep_sign_sum;
    err |= C.error;
  }
  S.prec_green_mean = events ? prec_sum / (double)events : 0.0;
  S.mean_sign = sign_sum / ((double)n_sweeps * n);
  S.ms_total = ms;
  if (stats) *stats = S;
  if (err) return fail(ctx, DQMC_EUNSTABLE, "singular matrix in the stabilisation");
  const double thr = ctx->opts.unstable_threshold;
  if (thr > 0.0 && (S.prec_green_max > thr || S.prec_phase_max > thr))
    return fail(ctx, DQMC_EUNSTABLE, "precision %.3e / phase %.3e above the threshold %.3e", S.prec_green_max,
                S.prec_phase_max, thr);
  return DQMC_OK;
}

dqmc_status dqmc_su2_greens(dqmc_su2_ctx* ctx, int32_t chain, int32_t fresh, double* out, int32_t out_is_device,
                            double* logabs_out, double* arg_out, double* phase_out) {
  if (!ctx || !ctx->chains_d) return fail(ctx, DQMC_ESTATE, "context not initialised");
  if (chain < 0 || chain >= (int)ctx->chains_h.size() || !out) return fail(ctx, DQMC_EINVAL, "bad chain or output");
  const int N = ctx->chains_h[chain].N;
  const size_t bytes = sizeof(double2) * (size_t)N * N;
  double2* dst = out_is_device ? reinterpret_cast<double2*>(out) : ctx->out_scratch;
  if (fresh)
    SU2_CUDA_TRY(ctx, dqmc::su2_launch_fresh(ctx->chains_d, (int)ctx->chains_h.size(), 1, chain, dst, ctx->smem,
                                             ctx->stream));
  else
    SU2_CUDA_TRY(ctx, dqmc::su2_launch_copy_green(ctx->chains_d, chain, dst, ctx->stream));
  if (!out_is_device)
    SU2_CUDA_TRY(ctx, cudaMemcpyAsync(out, ctx->out_scratch, bytes, cudaMemcpyDeviceToHost, ctx->stream));
  dqmc_status st = download(ctx);
  if (st) return st;
  const Su2Dev& C = ctx->chains_h[chain];
  if (C.error) return fail(ctx, DQMC_EUNSTABLE, "chain %d: singular matrix in the stabilisation", chain);
  if (logabs_out) *logabs_out = C.logabs;
  if (arg_out) *arg_out = C.arg;
  if (phase_out) { phase_out[0] = C.P.x; phase_out[1] = C.P.y; }
  return DQMC_OK;
}

dqmc_status dqmc_su2_measure(dqmc_su2_ctx* ctx, double* out, double* sign_sum, int64_t* n_meas, int32_t reset) {
  if (!ctx || !ctx->chains_d) return fail(ctx, DQMC_ESTATE, "context not initialised");
  dqmc_status st = download(ctx);
  if (st) return st;
  for (size_t c = 0; c < ctx->chains_h.size(); ++c) {
    const Su2Dev& C = ctx->chains_h[c];
    if (out)
      for (int q = 0; q < 10; ++q) out[c * 10 + q] = C.meas[q];
    if (sign_sum) sign_sum[c] = C.meas_sign;
    if (n_meas) n_meas[c] = C.n_meas;
  }
  if (reset) SU2_CUDA_TRY(ctx, dqmc::su2_launch_reset_stats(ctx->chains_d, (int)ctx->chains_h.size(), 1, ctx->stream));
  return DQMC_OK;
}

dqmc_status dqmc_su2_measure_tau(dqmc_su2_ctx* ctx, int32_t n_tau, double* out, double* prec_tau) {
  if (!ctx || !ctx->chains_d) return fail(ctx, DQMC_ESTATE, "context not initialised");
  if (!out) return fail(ctx, DQMC_EINVAL, "null output");
  const int nch = (int)ctx->chains_h.size();
  for (const Su2Dev& C : ctx->chains_h)
    if (n_tau < 0 || n_tau > C.L) return fail(ctx, DQMC_EINVAL, "n_tau must be in [0, L] of every chain");
  double2* a_d = nullptr;
  double* p_d = nullptr;
  const size_t na = (size_t)nch * (n_tau + 1);
  if (cudaMalloc((void**)&a_d, na * sizeof(double2)) != cudaSuccess ||
      cudaMalloc((void**)&p_d, (size_t)nch * 2 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(a_d);
    return fail(ctx, DQMC_ENOMEM, "tau measurement buffers");
  }
  std::vector<double> pr((size_t)nch * 2, 0.0);
  dqmc_status st = DQMC_OK;
  cudaError_t e = dqmc::su2_launch_tau(ctx->chains_d, nch, -1, n_tau, a_d, p_d, nullptr, nullptr, ctx->smem, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, a_d, na * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(pr.data(), p_d, pr.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
  if (e != cudaSuccess) st = fail(ctx, DQMC_ECUDA, "tau measurement: %s", cudaGetErrorString(e));
  if (!st) st = download(ctx);
  cudaFree(a_d);
  cudaFree(p_d);
  if (st) return st;
  double mean = 0.0, mx = 0.0;
  for (int c = 0; c < nch; ++c) {
    if (ctx->chains_h[c].error) return fail(ctx, DQMC_EUNSTABLE, "chain %d: singular matrix in the tau measurement", c);
    mean += pr[2 * c] / nch;
    mx = std::max(mx, pr[2 * c + 1]);
  }
  if (prec_tau) { prec_tau[0] = mean; prec_tau[1] = mx; }
  return DQMC_OK;
}

dqmc_status dqmc_su2_greens_displaced(dqmc_su2_ctx* ctx, int32_t chain, int32_t tau, double* out_t0, double* out_0t) {
  if (!ctx || !ctx->chains_d) return fail(ctx, DQMC_ESTATE, "context not initialised");
  if (chain < 0 || chain >= (int)ctx->chains_h.size() || !out_t0 || !out_0t)
    return fail(ctx, DQMC_EINVAL, "bad chain or output");
  const Su2Dev& H = ctx->chains_h[chain];
  if (tau < 0 || tau > H.L) return fail(ctx, DQMC_EINVAL, "tau must be in [0, L]");
  const size_t nn = (size_t)H.N * H.N;
  double2* g_d = nullptr;
  if (cudaMalloc((void**)&g_d, 2 * nn * sizeof(double2)) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, DQMC_ENOMEM, "displaced Green function buffers");
  }
  dqmc_status st = DQMC_OK;
  cudaError_t e = dqmc::su2_launch_tau(ctx->chains_d, (int)ctx->chains_h.size(), chain, tau, nullptr, nullptr, g_d,
                                       g_d + nn, ctx->smem, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out_t0, g_d, nn * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out_0t, g_d + nn, nn * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream);
  if (e != cudaSuccess) st = fail(ctx, DQMC_ECUDA, "displaced Green functions: %s", cudaGetErrorString(e));
  if (!st) st = download(ctx);
  cudaFree(g_d);
  if (st) return st;
  if (ctx->chains_h[chain].error) return fail(ctx, DQMC_EUNSTABLE, "chain %d: singular matrix", chain);
  return DQMC_OK;
}

dqmc_status dqmc_su2_measure_corr(dqmc_su2_ctx* ctx, const int32_t* pair_class, const int32_t* n_class, double* out,
                                  double* phase) {
  if (!ctx || !ctx->chains_d) return fail(ctx, DQMC_ESTATE, "context not initialised");
  if (!pair_class || !n_class || !out || !phase) return fail(ctx, DQMC_EINVAL, "null argument");
  const int nm = (int)ctx->models.size(), nch = (int)ctx->chains_h.size();
  // CSR lists of every model's pair classes (pairs in row-major order of (x, y))
  std::vector<std::vector<int>> off(nm), prs(nm);
  size_t cls_off = 0;
  int max_cls = 1;
  for (int m = 0; m < nm; ++m) {
    const int N = ctx->models[m].n_sites, nc = n_class[m];
    if (nc < 1) return fail(ctx, DQMC_EINVAL, "model %d: n_class must be >= 1", m);
    max_cls = std::max(max_cls, nc);
    const int32_t* cls = pair_class + cls_off;
    cls_off += (size_t)N * N;
    std::vector<int> cnt(nc + 1, 0);
    for (int e = 0; e < N * N; ++e) {
      if (cls[e] < -1 || cls[e] >= nc) return fail(ctx, DQMC_EINVAL, "model %d: pair class %d out of range", m, cls[e]);
      if (cls[e] >= 0) ++cnt[cls[e] + 1];
    }
    for (int k = 0; k < nc; ++k) cnt[k + 1] += cnt[k];
    off[m] = cnt;
    prs[m].assign((size_t)cnt[nc] + 1, 0);
    std::vector<int> fill(cnt.begin(), cnt.end() - 1);
    for (int e = 0; e < N * N; ++e)
      if (cls[e] >= 0) prs[m][fill[cls[e]]++] = e;
  }
  std::vector<void*> tmp;
  auto release = [&]() { for (void* q : tmp) cudaFree(q); };
  auto up = [&](const void* src, size_t bytes) -> void* {
    void* d = nullptr;
    if (cudaMalloc(&d, bytes) != cudaSuccess) return nullptr;
    tmp.push_back(d);
    if (cudaMemcpy(d, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess) return nullptr;
    return d;
  };
  std::vector<const int*> offd(nm), prd(nm), coff(nch), cpr(nch);
  std::vector<int> cnc(nch);
  for (int m = 0; m < nm; ++m) {
    offd[m] = static_cast<const int*>(up(off[m].data(), off[m].size() * sizeof(int)));
    prd[m] = static_cast<const int*>(up(prs[m].data(), prs[m].size() * sizeof(int)));
    if (!offd[m] || !prd[m]) { release(); return fail(ctx, DQMC_ENOMEM, "class lists"); }
  }
  for (int c = 0; c < nch; ++c) {
    const int m = ctx->chain_model[c];
    coff[c] = offd[m];
    cpr[c] = prd[m];
    cnc[c] = n_class[m];
  }
  const int* const* coff_d = static_cast<const int* const*>(up(coff.data(), nch * sizeof(int*)));
  const int* const* cpr_d = static_cast<const int* const*>(up(cpr.data(), nch * sizeof(int*)));
  const int* cnc_d = static_cast<const int*>(up(cnc.data(), nch * sizeof(int)));
  const size_t nout = (size_t)nch * max_cls * 4;
  double2* out_d = nullptr;
  if (!coff_d || !cpr_d || !cnc_d || cudaMalloc((void**)&out_d, nout * sizeof(double2)) != cudaSuccess) {
    cudaGetLastError();
    release();
    return fail(ctx, DQMC_ENOMEM, "correlation buffers");
  }
  tmp.push_back(out_d);
  dqmc_status st = DQMC_OK;
  cudaError_t e = dqmc::su2_launch_corr(ctx->chains_d, nch, coff_d, cpr_d, cnc_d, max_cls, out_d, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, out_d, nout * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream);
  if (e != cudaSuccess) st = fail(ctx, DQMC_ECUDA, "correlations: %s", cudaGetErrorString(e));
  if (!st) st = download(ctx);
  release();
  if (st) return st;
  for (int c = 0; c < nch; ++c) {
    phase[2 * c] = ctx->chains_h[c].P.x;
    phase[2 * c + 1] = ctx->chains_h[c].P.y;
  }
  return DQMC_OK;
}

dqmc_status dqmc_su2_get_fields(dqmc_su2_ctx* ctx, int8_t* out, uint64_t* sweep_counter) {
  if (!ctx || !ctx->chains_d) return fail(ctx, DQMC_ESTATE, "context not initialised");
  if (out) {
    size_t off = 0;
    for (const Su2Dev& C : ctx->chains_h) {
      SU2_CUDA_TRY(ctx, cudaMemcpyAsync(out + off, C.fields, (size_t)C.L * C.MV, cudaMemcpyDeviceToHost, ctx->stream));
      off += (size_t)C.L * C.MV;
    }
    SU2_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  }
  if (sweep_counter) *sweep_counter = ctx->sweep_counter;
  return DQMC_OK;
}

dqmc_status dqmc_su2_set_fields(dqmc_su2_ctx* ctx, const int8_t* in, uint64_t sweep_counter) {
  if (!ctx || !ctx->chains_d) return fail(ctx, DQMC_ESTATE, "context not initialised");
  if (!in) return fail(ctx, DQMC_EINVAL, "null fields");
  size_t off = 0;
  for (const Su2Dev& C : ctx->chains_h) {
    dqmc_status st = check_fields(ctx, in + off, C.L, C.N, C.MV);
    if (st) return st;
    off += (size_t)C.L * C.MV;
  }
  off = 0;
  for (const Su2Dev& C : ctx->chains_h) {
    SU2_CUDA_TRY(ctx, cudaMemcpyAsync(C.fields, in + off, (size_t)C.L * C.MV, cudaMemcpyHostToDevice, ctx->stream));
    off += (size_t)C.L * C.MV;
  }
  ctx->sweep_counter = sweep_counter;
  return refill(ctx);
}

const char* dqmc_su2_last_error(const dqmc_su2_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

void dqmc_su2_destroy(dqmc_su2_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  else cudaDeviceSynchronize();
  for (void* p : ctx->allocs) cudaFree(p);
  if (ctx->chains_d) cudaFree(ctx->chains_d);
  if (ctx->out_scratch) cudaFree(ctx->out_scratch);
  if (ctx->ev0) cudaEventDestroy(ctx->ev0);
  if (ctx->ev1) cudaEventDestroy(ctx->ev1);
  delete ctx;
}

}  // extern "C"
