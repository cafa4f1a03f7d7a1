// Host side of the C ABI declared in include/dqmc.h: validation, model set-up
// (the exponentials exp(-+dtau K) of Sec. 3.1, Op_set), the device arena of
// every chain, and the launches of the kernels in dqmc_kernels.cu.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <numeric>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "../../include/dqmc.h"
#include "dqmc_internal.h"
#include "dqmc_linalg_host.h"

using dqmc::ChainDev;
using dqmc::host::expm_symmetric;
using dqmc::host::symmetric_eigen;

namespace {

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Site count from which chains of a DQMC_PREC_MIXED_TC context run their N^3
// products on the tensor cores (smaller ones keep the float-pair SIMT tiles).
constexpr int kDefaultTcMinSites = 96;
int tc_min_sites(const dqmc_run_opts& o) { return o.tc_min_sites > 0 ? o.tc_min_sites : kDefaultTcMinSites; }


struct ModelHost {
  dqmc_model_desc d;
  int ld = 0;
  double cscale = 0.0;
  std::vector<double> hopping, vsign;
  std::vector<int> site;
  std::vector<double> eigval[dqmc::kMaxFlavors], eigvec[dqmc::kMaxFlavors];
  // device
  double *K = nullptr, *E = nullptr, *Einv = nullptr, *ident = nullptr, *vsign_d = nullptr;
  float *E32 = nullptr, *Einv32 = nullptr;
  float *Edd = nullptr, *Einvdd = nullptr;  // (hi, lo) pairs
  int* site_d = nullptr;
  // split-product planes of the constant propagators (tensor-core products only)
  void* cpl[dqmc::kMaxFlavors][5] = {};
  int* cex[dqmc::kMaxFlavors][5] = {};
  CUtensorMap tmc[dqmc::kMaxFlavors][5] = {};
};

}  // namespace

struct dqmc_ctx {
  std::string err;
  cudaStream_t stream = nullptr;
  dqmc_run_opts opts{};
  int nfl = 0;
  std::vector<ModelHost> models;
  std::vector<int> chain_model;
  std::vector<ChainDev> chains_h;
  ChainDev* chains_d = nullptr;
  int* order_d = nullptr;
  unsigned char* arena = nullptr;
  std::vector<void*> model_allocs;
  int kprec = 0;          // working-G storage: 0 double, 1 float, 2 float pairs (the sweep, fresh-G and
                          // wrapped-G kernels are chosen by opts.precision: 3 adds the tensor cores)
  size_t smem = 0;        // dynamic shared memory of the fresh-G / gradient kernels
  size_t smem_sweep = 0;  // ... of the sweep kernel (plus the delayed vectors when they fit)
  int ab_smem = 0;
  uint64_t sweep_counter = 0;
  int maxN = 0, maxld = 0, maxMV = 0;
  double* scratch = nullptr;  // [nfl][maxN][maxN] FP64 for dqmc_greens
  double* tau_work = nullptr;  // [n_chains][nfl][4][maxN][maxld] FP64 for dqmc_measure_tau (on first use)
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

namespace {

dqmc_status fail(dqmc_ctx* ctx, dqmc_status st, const char* fmt, ...) {
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

#define CUDA_TRY(ctx, expr)                                                                      \
  do {                                                                                           \
    cudaError_t e_ = (expr);                                                                     \
    if (e_ != cudaSuccess) return fail(ctx, DQMC_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
  } while (0)

dqmc_status validate_model(dqmc_ctx* ctx, const dqmc_model_desc& m, int idx) {
  if (m.n_sites < 1 || m.n_flavors < 1 || m.n_flavors > dqmc::kMaxFlavors)
    return fail(ctx, DQMC_EINVAL, "model %d: n_sites must be >= 1 and n_flavors 1 or 2", idx);
  if (!m.hopping || !m.vertex_site || !m.vertex_sign) return fail(ctx, DQMC_EINVAL, "model %d: null array", idx);
  if (m.n_vertices < 1 || m.n_vertices > m.n_sites)
    return fail(ctx, DQMC_EINVAL, "model %d: n_vertices must be in [1, n_sites]", idx);
  if (m.field_type != DQMC_FIELD_ISING && m.field_type != DQMC_FIELD_HS4)
    return fail(ctx, DQMC_EINVAL, "model %d: unknown field_type %d", idx, m.field_type);
  if (!(m.dtau > 0.0) || !std::isfinite(m.dtau)) return fail(ctx, DQMC_EINVAL, "model %d: dtau must be > 0", idx);
  if (!(m.U >= 0.0) || !std::isfinite(m.U)) return fail(ctx, DQMC_EINVAL, "model %d: U must be >= 0", idx);
  if (m.L < 1 || m.n_wrap < 1 || m.L % m.n_wrap != 0)
    return fail(ctx, DQMC_EINVAL, "model %d: L must be a positive multiple of n_wrap", idx);
  const int N = m.n_sites;
  std::vector<char> seen(N, 0);
  for (int k = 0; k < m.n_vertices; ++k) {
    const int s = m.vertex_site[k];
    if (s < 0 || s >= N || seen[s]) return fail(ctx, DQMC_EINVAL, "model %d: vertex sites must be distinct in [0,N)", idx);
    seen[s] = 1;
  }
  for (int f = 0; f < m.n_flavors; ++f) {
    const double* K = m.hopping + (size_t)f * N * N;
    double mx = 0.0;
    for (int i = 0; i < N * N; ++i) {
      if (!std::isfinite(K[i])) return fail(ctx, DQMC_EINVAL, "model %d: non-finite hopping", idx);
      mx = std::max(mx, std::fabs(K[i]));
    }
    for (int i = 0; i < N; ++i)
      for (int j = i + 1; j < N; ++j)
        if (std::fabs(K[(size_t)i * N + j] - K[(size_t)j * N + i]) > 1e-12 * (1.0 + mx))
          return fail(ctx, DQMC_EINVAL, "model %d: hopping matrix of flavor %d is not symmetric", idx, f);
    for (int k = 0; k < m.n_vertices; ++k)
      if (!std::isfinite(m.vertex_sign[(size_t)f * m.n_vertices + k]))
        return fail(ctx, DQMC_EINVAL, "model %d: non-finite vertex_sign", idx);
  }
  return DQMC_OK;
}

template <typename T>
dqmc_status upload(dqmc_ctx* ctx, T** dst, const T* src, size_t n) {
  void* p = nullptr;
  CUDA_TRY(ctx, cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)));
  ctx->model_allocs.push_back(p);
  if (n) CUDA_TRY(ctx, cudaMemcpy(p, src, n * sizeof(T), cudaMemcpyHostToDevice));
  *dst = (T*)p;
  return DQMC_OK;
}

// The driver's tensor-map encoder, through the runtime's entry-point query (the
// library does not link against the driver library).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// Tensor map of a digit-plane buffer of `bytes` bytes for the split products:
// the 4D view [blocks][kPlaneDigits][rows][kPlaneK] of bf16 (k innermost,
// contiguous) with a box of one whole block, so that a tiled copy at block
// coordinate b moves the b-th block's bytes unchanged.  0 on success.
int encode_plane_map(CUtensorMap* tm, void* base, int rows, size_t bytes) {
  const PFN_cuTensorMapEncodeTiled_v12000 fn = tensor_map_encoder();
  if (!fn) return 1;
  const uint64_t row_bytes = (uint64_t)dqmc::kPlaneK * 2;
  const uint64_t blk = (uint64_t)dqmc::kPlaneDigits * rows * row_bytes;
  if (bytes < blk || (reinterpret_cast<uintptr_t>(base) & 15) != 0) return 2;
  const cuuint64_t dims[4] = {(cuuint64_t)dqmc::kPlaneK, (cuuint64_t)rows, (cuuint64_t)dqmc::kPlaneDigits,
                              (cuuint64_t)(bytes / blk)};
  const cuuint64_t strides[3] = {row_bytes, (cuuint64_t)rows * row_bytes, blk};
  const cuuint32_t box[4] = {(cuuint32_t)dqmc::kPlaneK, (cuuint32_t)rows, (cuuint32_t)dqmc::kPlaneDigits, 1u};
  const cuuint32_t es[4] = {1u, 1u, 1u, 1u};
  const CUresult r = fn(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, base, dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 0 : 3;
}

size_t pad_to(size_t n, size_t q) { return (n + q - 1) / q * q; }

dqmc_status setup_model(dqmc_ctx* ctx, ModelHost& M) {
  const dqmc_model_desc& d = M.d;
  const int N = d.n_sites, nfl = d.n_flavors;
  const int ld = (int)align_up(N, 4);
  M.ld = ld;
  M.cscale = (d.field_type == DQMC_FIELD_ISING) ? std::acosh(std::exp(0.5 * d.dtau * d.U)) : std::sqrt(0.5 * d.dtau * d.U);
  M.hopping.assign(d.hopping, d.hopping + (size_t)nfl * N * N);
  M.vsign.assign(d.vertex_sign, d.vertex_sign + (size_t)nfl * d.n_vertices);
  M.site.assign(d.vertex_site, d.vertex_site + d.n_vertices);
  M.d.hopping = nullptr;
  M.d.vertex_site = nullptr;
  M.d.vertex_sign = nullptr;
  std::vector<double> K((size_t)nfl * N * ld, 0.0), E((size_t)nfl * N * ld, 0.0), Ei((size_t)nfl * N * ld, 0.0);
  std::vector<float> E32((size_t)nfl * N * ld, 0.f), Ei32((size_t)nfl * N * ld, 0.f);
  std::vector<float> Edd((size_t)2 * nfl * N * ld, 0.f), Eidd((size_t)2 * nfl * N * ld, 0.f);
  for (int f = 0; f < nfl; ++f) {
    std::vector<double> Kf(M.hopping.begin() + (size_t)f * N * N, M.hopping.begin() + (size_t)(f + 1) * N * N);
    symmetric_eigen(N, Kf, M.eigval[f], M.eigvec[f]);
    const std::vector<double> Ef = expm_symmetric(N, M.eigval[f], M.eigvec[f], -d.dtau);
    const std::vector<double> Eif = expm_symmetric(N, M.eigval[f], M.eigvec[f], +d.dtau);
    for (size_t q = 0; q < Ef.size(); ++q)
      if (!std::isfinite(Ef[q]) || !std::isfinite(Eif[q]))
        return fail(ctx, DQMC_EINVAL, "exp(-+dtau K) of flavor %d is not finite (dtau * |K| too large)", f);
    for (int i = 0; i < N; ++i)
      for (int j = 0; j < N; ++j) {
        const size_t o = (size_t)f * N * ld + (size_t)i * ld + j;
        K[o] = Kf[(size_t)i * N + j];
        E[o] = Ef[(size_t)i * N + j];
        Ei[o] = Eif[(size_t)i * N + j];
        E32[o] = (float)E[o];
        Ei32[o] = (float)Ei[o];
        Edd[2 * o] = E32[o];
        Edd[2 * o + 1] = (float)(E[o] - (double)E32[o]);
        Eidd[2 * o] = Ei32[o];
        Eidd[2 * o + 1] = (float)(Ei[o] - (double)Ei32[o]);
      }
  }
  std::vector<double> ident((size_t)2 * N * ld + ld, 0.0);
  for (int i = 0; i < N; ++i) {
    ident[(size_t)i * ld + i] = 1.0;
    ident[(size_t)N * ld + (size_t)i * ld + i] = 1.0;
    ident[(size_t)2 * N * ld + i] = 1.0;
  }
  dqmc_status st;
  if ((st = upload(ctx, &M.K, K.data(), K.size()))) return st;
  if ((st = upload(ctx, &M.E, E.data(), E.size()))) return st;
  if ((st = upload(ctx, &M.Einv, Ei.data(), Ei.size()))) return st;
  if ((st = upload(ctx, &M.E32, E32.data(), E32.size()))) return st;
  if ((st = upload(ctx, &M.Einv32, Ei32.data(), Ei32.size()))) return st;
  if ((st = upload(ctx, &M.Edd, Edd.data(), Edd.size()))) return st;
  if ((st = upload(ctx, &M.Einvdd, Eidd.data(), Eidd.size()))) return st;
  if ((st = upload(ctx, &M.ident, ident.data(), ident.size()))) return st;
  if ((st = upload(ctx, &M.site_d, M.site.data(), M.site.size()))) return st;
  if ((st = upload(ctx, &M.vsign_d, M.vsign.data(), M.vsign.size()))) return st;
  if (ctx->opts.precision == DQMC_PREC_MIXED_TC && N >= tc_min_sites(ctx->opts)) {
    // digit planes of e^-dtau K and e^+dtau K as the left and right factors of the
    // wraps and of the B chain, split once per model (Sec. 3.1: the hopping
    // propagator is a constant of the model)
    struct { int which, right, tr; bool inv; } sets[5] = {{dqmc::kCpEA, 0, 0, false},
                                                           {dqmc::kCpEtA, 0, 1, false},
                                                           {dqmc::kCpEiA, 0, 0, true},
                                                           {dqmc::kCpEiB, 1, 0, true},
                                                           {dqmc::kCpEB, 1, 0, false}};
    const size_t mat = (size_t)N * ld;
    for (int f = 0; f < nfl; ++f)
      for (const auto& q : sets) {
        void* p = nullptr;
        int* e = nullptr;
        CUDA_TRY(ctx, cudaMalloc(&p, dqmc::const_plane_bytes(N, q.right)));
        ctx->model_allocs.push_back(p);
        CUDA_TRY(ctx, cudaMalloc((void**)&e, sizeof(int) * dqmc::const_plane_exps(N, q.right)));
        ctx->model_allocs.push_back(e);
        const float* X = (q.inv ? M.Einvdd : M.Edd) + 2 * f * mat;
        CUDA_TRY(ctx, dqmc::launch_const_planes(X, N, ld, q.right, q.tr, p, e, ctx->stream));
        M.cpl[f][q.which] = p;
        M.cex[f][q.which] = e;
        const int em = encode_plane_map(&M.tmc[f][q.which], p, q.right ? dqmc::kPlaneRowsB : dqmc::kPlaneRowsA,
                                        dqmc::const_plane_bytes(N, q.right));
        if (em) return fail(ctx, DQMC_ECUDA, "tensor map of the constant digit planes (code %d)", em);
      }
  }
  return DQMC_OK;
}

// Per-chain device memory, carved from one arena.  Returns the bytes needed
// (ptrs filled when base != nullptr).
size_t chain_layout(const ModelHost& M, int precision, int delay_k, unsigned char* base, ChainDev* C,
                    int tc_min = 1) {
  const int N = M.d.n_sites, ld = M.ld, nfl = M.d.n_flavors, nst = M.d.L / M.d.n_wrap;
  const size_t rs = precision == DQMC_PREC_FP32 ? sizeof(float) : sizeof(double);  // FP64 or float pairs
  size_t off = 0;
  auto take = [&](size_t bytes) -> unsigned char* {
    off = align_up(off, 256);
    unsigned char* p = base ? base + off : nullptr;
    off += bytes;
    return p;
  };
  unsigned char* p = take((size_t)M.d.L * M.d.n_vertices);
  if (C) C->fields = (int8_t*)p;
  for (int s = 0; s < nfl; ++s) {
    p = take((size_t)N * ld * rs);
    if (C) C->G[s] = p;
    p = take((size_t)N * ld * rs);
    if (C) C->Gtmp[s] = p;
    p = take((size_t)delay_k * ld * rs);
    if (C) C->dA[s] = p;
    p = take((size_t)delay_k * ld * rs);
    if (C) C->dB[s] = p;
    p = take((size_t)(nst + 1) * dqmc::slot_stride(N, ld) * sizeof(double));
    if (C) C->slots[s] = (double*)p;
    p = take((size_t)(nst + 1) * sizeof(int));
    if (C) C->slot_detq[s] = (int*)p;
    p = take(dqmc::work_elems(N, ld) * sizeof(double));
    if (C) C->work[s] = (double*)p;
    p = take((size_t)2 * ld * sizeof(int));
    if (C) C->iwork[s] = (int*)p;
    if (precision == DQMC_PREC_MIXED_TC && N >= tc_min) {
      // BF16 digit planes of the split tensor-core products (N x N x N at most)
      p = take(dqmc::plane_bytes(N, N));
      if (C) C->planes[s] = p;
    }
  }
  return align_up(off, 256);
}

void fill_model_fields(const ModelHost& M, ChainDev& C) {
  const dqmc_model_desc& d = M.d;
  C.N = d.n_sites;
  C.ld = M.ld;
  C.nfl = d.n_flavors;
  C.MV = d.n_vertices;
  C.L = d.L;
  C.nw = d.n_wrap;
  C.ft = d.field_type;
  C.dtau = d.dtau;
  C.U = d.U;
  C.cscale = M.cscale;
  const size_t mat = (size_t)d.n_sites * M.ld;
  for (int s = 0; s < d.n_flavors; ++s) {
    C.K[s] = M.K + s * mat;
    C.E[s] = M.E + s * mat;
    C.Einv[s] = M.Einv + s * mat;
    C.E32[s] = M.E32 + s * mat;
    C.Einv32[s] = M.Einv32 + s * mat;
    C.Edd[s] = M.Edd + 2 * s * mat;
    C.Einvdd[s] = M.Einvdd + 2 * s * mat;
    for (int q = 0; q < 5; ++q) {
      C.cpl[s][q] = M.cpl[s][q];
      C.cex[s][q] = M.cex[s][q];
      C.tm_cp[s][q] = M.tmc[s][q];
    }
  }
  C.site = M.site_d;
  C.vsign = M.vsign_d;
  C.ident = M.ident;
}

dqmc_status sync_check(dqmc_ctx* ctx) {
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  CUDA_TRY(ctx, cudaGetLastError());
  return DQMC_OK;
}

dqmc_status download_chains(dqmc_ctx* ctx) {
  CUDA_TRY(ctx, cudaMemcpyAsync(ctx->chains_h.data(), ctx->chains_d, sizeof(ChainDev) * ctx->chains_h.size(),
                                cudaMemcpyDeviceToHost, ctx->stream));
  return sync_check(ctx);
}

// DQMC_ETIMEOUT with the first wait that gave up in each flavor of chain C.
dqmc_status timeout_message(dqmc_ctx* ctx, const ChainDev& C) {
  std::string m;
  bool misaligned = false;
  for (int s = 0; s < C.nfl; ++s) {
    const int* w = C.wait_where[s];
    misaligned = misaligned || w[0] == 9;
    char b[200];
    snprintf(b, sizeof(b), "; flavor %d: kind %d at chunk %d of %d in product %d (barrier %08x %08x)", s, w[0], w[1],
             w[2], w[3], (unsigned)w[5], (unsigned)w[4]);
    m += b;
  }
  if (misaligned)
    return fail(ctx, DQMC_ECUDA, "chain %u: staging buffers of the tensor-core products not 128-byte aligned%s",
                C.chain_id, m.c_str());
  return fail(ctx, DQMC_ETIMEOUT, "chain %u: a bounded wait of the tensor-core products gave up%s", C.chain_id,
              m.c_str());
}

// Fields in place -> left chain, G(0), sign of every chain.
dqmc_status initial_fill(dqmc_ctx* ctx) {
  const int n = (int)ctx->chains_h.size();
  dqmc::set_smem_bytes(ctx->smem);
  CUDA_TRY(ctx, dqmc::launch_fresh_green(ctx->chains_d, n, ctx->nfl, ctx->opts.precision, 1, nullptr, -1,
                                         ctx->stream));
  CUDA_TRY(ctx, dqmc::launch_finalize_init(ctx->chains_d, n, ctx->stream));
  dqmc_status st = download_chains(ctx);
  if (st) return st;
  for (const ChainDev& C : ctx->chains_h) {
    if (C.error & 2) return timeout_message(ctx, C);
    if (C.error) return fail(ctx, DQMC_EUNSTABLE, "chain %u: singular matrix in the stabilisation", C.chain_id);
  }
  return DQMC_OK;
}

}  // namespace

extern "C" {

dqmc_status dqmc_init(const dqmc_model_desc* models, int32_t n_models, const int32_t* chain_model, int32_t n_chains,
                      const int8_t* fields_or_null, const dqmc_run_opts* opts, void* cuda_stream, dqmc_ctx** out) {
  if (!out) return DQMC_EINVAL;
  *out = nullptr;
  std::unique_ptr<dqmc_ctx> ctx(new dqmc_ctx());
  dqmc_ctx* c = ctx.get();
  if (!models || n_models < 1 || !chain_model || n_chains < 1 || !opts) {
    *out = ctx.release();
    return fail(*out, DQMC_EINVAL, "null argument or empty model/chain list");
  }
  c->opts = *opts;
  c->kprec = opts->precision == DQMC_PREC_MIXED_TC ? DQMC_PREC_MIXED : opts->precision;
  if (opts->precision < DQMC_PREC_FP64 || opts->precision > DQMC_PREC_MIXED_TC) {
    *out = ctx.release();
    return fail(*out, DQMC_EINVAL, "unknown precision %d", opts->precision);
  }
  if (opts->spin_limit < 0 || opts->tc_min_sites < 0) {
    *out = ctx.release();
    return fail(*out, DQMC_EINVAL, "spin_limit and tc_min_sites must be >= 0");
  }
  if (opts->stab_svd != 0 && (opts->stab_svd != 1 || opts->precision != DQMC_PREC_FP64)) {
    *out = ctx.release();
    return fail(*out, DQMC_EINVAL, "stab_svd must be 0, or 1 with DQMC_PREC_FP64");
  }
  if (opts->dd_tile != 0 && opts->dd_tile != 3 && opts->dd_tile != 4) {
    *out = ctx.release();
    return fail(*out, DQMC_EINVAL, "dd_tile must be 0, 3 or 4");
  }
  if (opts->delay_k < 1 || opts->delay_k > 64) {
    *out = ctx.release();
    return fail(*out, DQMC_EINVAL, "delay_k must be in [1, 64]");
  }
  c->stream = (cudaStream_t)cuda_stream;
  dqmc_status st = DQMC_OK;
  for (int m = 0; m < n_models && !st; ++m) st = validate_model(c, models[m], m);
  for (int m = 1; m < n_models && !st; ++m)
    if (models[m].n_flavors != models[0].n_flavors) st = fail(c, DQMC_EINVAL, "all models need the same n_flavors");
  for (int i = 0; i < n_chains && !st; ++i)
    if (chain_model[i] < 0 || chain_model[i] >= n_models) st = fail(c, DQMC_EINVAL, "chain_model[%d] out of range", i);
  if (st) {
    *out = ctx.release();
    return st;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    *out = ctx.release();
    return fail(*out, DQMC_ECUDA, "no CUDA device available (the library has no CPU path)");
  }
  c->nfl = models[0].n_flavors;
  c->models.resize(n_models);
  for (int m = 0; m < n_models && !st; ++m) {
    c->models[m].d = models[m];
    st = setup_model(c, c->models[m]);
    c->maxN = std::max(c->maxN, models[m].n_sites);
    c->maxld = std::max(c->maxld, c->models[m].ld);
    c->maxMV = std::max(c->maxMV, models[m].n_vertices);
  }
  if (st) {
    *out = ctx.release();
    return st;
  }
  c->chain_model.assign(chain_model, chain_model + n_chains);
  // arena
  std::vector<size_t> offs(n_chains);
  size_t total = 0;
  for (int i = 0; i < n_chains; ++i) {
    offs[i] = total;
    total += chain_layout(c->models[chain_model[i]], opts->precision, opts->delay_k, nullptr, nullptr,
                          tc_min_sites(*opts));
  }
  if (cudaMalloc((void**)&c->arena, total) != cudaSuccess) {
    *out = ctx.release();
    return fail(*out, DQMC_ENOMEM, "device arena of %zu bytes", total);
  }
  cudaMemsetAsync(c->arena, 0, total, c->stream);
  c->chains_h.assign(n_chains, ChainDev{});
  size_t foff = 0;
  for (int i = 0; i < n_chains; ++i) {
    ChainDev& C = c->chains_h[i];
    const ModelHost& M = c->models[chain_model[i]];
    chain_layout(M, opts->precision, opts->delay_k, c->arena + offs[i], &C, tc_min_sites(*opts));
    fill_model_fields(M, C);
    for (int s = 0; s < M.d.n_flavors; ++s) {
      if (!C.planes[s]) continue;
      // the scratch planes: the left operand's blocks first, the right operand's
      // after them (the offset the kernels use)
      const size_t N = (size_t)M.d.n_sites, kp = pad_to(N, dqmc::kPlaneK);
      const size_t bytesA = (size_t)dqmc::kPlaneDigits * pad_to(N, dqmc::kPlaneRowsA) * kp * 2;
      const size_t bytesB = (size_t)dqmc::kPlaneDigits * pad_to(N, dqmc::kPlaneRowsB) * kp * 2;
      int em = encode_plane_map(&C.tm_pl[s][0], C.planes[s], dqmc::kPlaneRowsA, bytesA);
      if (!em)
        em = encode_plane_map(&C.tm_pl[s][1], static_cast<unsigned char*>(C.planes[s]) + bytesA, dqmc::kPlaneRowsB,
                              bytesB);
      if (em) {
        *out = ctx.release();
        return fail(*out, DQMC_ECUDA, "tensor map of the digit-plane scratch (code %d)", em);
      }
    }
    C.chain_id = (uint32_t)i;
    C.sign = 1;
    C.wait_cycles = opts->spin_limit;
    C.dd_tile = opts->dd_tile;
    C.test_stall = opts->test_stall;
    C.stab_svd = opts->stab_svd;
    if (fields_or_null) {
      const size_t nf = (size_t)M.d.L * M.d.n_vertices;
      for (size_t q = 0; q < nf; ++q) {
        const int8_t f = fields_or_null[foff + q];
        const bool ok = (M.d.field_type == DQMC_FIELD_ISING) ? (f == 1 || f == -1)
                                                             : (f == 1 || f == -1 || f == 2 || f == -2);
        if (!ok) {
          *out = ctx.release();
          return fail(*out, DQMC_EINVAL, "chain %d: invalid field value %d", i, (int)f);
        }
      }
      cudaMemcpyAsync(C.fields, fields_or_null + foff, nf, cudaMemcpyHostToDevice, c->stream);
      foff += nf;
    }
  }
  *out = ctx.release();
  c = *out;
  CUDA_TRY(c, cudaMalloc((void**)&c->chains_d, sizeof(ChainDev) * n_chains));
  CUDA_TRY(c, cudaMemcpyAsync(c->chains_d, c->chains_h.data(), sizeof(ChainDev) * n_chains, cudaMemcpyHostToDevice,
                              c->stream));
  // heavy chains first (cost ~ L N^3)
  std::vector<int> order(n_chains);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    const auto& A = c->chains_h[a];
    const auto& B = c->chains_h[b];
    return (double)A.L * A.N * A.N * A.N > (double)B.L * B.N * B.N * B.N;
  });
  CUDA_TRY(c, cudaMalloc((void**)&c->order_d, sizeof(int) * n_chains));
  CUDA_TRY(c, cudaMemcpyAsync(c->order_d, order.data(), sizeof(int) * n_chains, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMalloc((void**)&c->scratch, sizeof(double) * c->nfl * c->maxN * c->maxN));
  CUDA_TRY(c, cudaEventCreate(&c->ev0));
  CUDA_TRY(c, cudaEventCreate(&c->ev1));
  {
    // the split tensor-core products stage their operands in a region of the
    // dynamic shared memory; in the sweep it doubles as the delayed vectors A, B,
    // kept in shared memory when they fit beside the rest
    const int umma = opts->precision == DQMC_PREC_MIXED_TC;
    const size_t base = dqmc::sweep_smem_bytes(c->maxN, c->maxld, c->maxMV, opts->delay_k, opts->precision);
    const size_t rs = c->kprec == DQMC_PREC_FP32 ? sizeof(float) : sizeof(double);
    const size_t ab = (size_t)2 * opts->delay_k * c->maxld * rs;
    c->smem = base + (umma ? dqmc::smem_tail(0, umma) : 0);
    c->ab_smem = (base + dqmc::smem_tail(ab, umma) <= 200 * 1024) ? 1 : 0;
    c->smem_sweep = base + dqmc::smem_tail(c->ab_smem ? ab : 0, umma);
    if (umma) {
      // every CTA of these kernels holds half of the SM's tensor
      // memory (256 of 512 columns): at least 78 KB of shared memory per CTA keeps
      // three of them from sharing an SM, so an allocation never waits
      c->smem = std::max<size_t>(c->smem, 78 * 1024);
      c->smem_sweep = std::max<size_t>(c->smem_sweep, 78 * 1024);
    }
  }
  if (!fields_or_null) CUDA_TRY(c, dqmc::launch_init_fields(c->chains_d, n_chains, opts->seed, 0, 0, c->stream));
  return initial_fill(c);
}

dqmc_status dqmc_sweep(dqmc_ctx* ctx, int32_t n_sweeps, dqmc_sweep_stats* stats) {
  if (!ctx) return DQMC_EINVAL;
  if (n_sweeps < 0) return fail(ctx, DQMC_EINVAL, "n_sweeps < 0");
  const int n = (int)ctx->chains_h.size();
  CUDA_TRY(ctx, dqmc::launch_reset_stats(ctx->chains_d, n, ctx->stream));
  if (stats) CUDA_TRY(ctx, cudaEventRecord(ctx->ev0, ctx->stream));
  dqmc::SweepParams P{};
  P.seed = ctx->opts.seed;
  P.delay_k = ctx->opts.delay_k;
  P.measure = ctx->opts.measure;
  P.meas_first = ctx->opts.meas_first;
  P.meas_last = ctx->opts.meas_last;
  P.n_chains = n;
  P.ab_smem = ctx->ab_smem;
  P.order = ctx->order_d;
  for (int i = 0; i < n_sweeps; ++i) {
    P.sweep = ctx->sweep_counter++;
    CUDA_TRY(ctx, dqmc::launch_sweep(ctx->chains_d, P, ctx->nfl, ctx->opts.precision, ctx->smem_sweep, ctx->stream));
  }
  if (!stats) return DQMC_OK;
  CUDA_TRY(ctx, cudaEventRecord(ctx->ev1, ctx->stream));
  dqmc_status st = download_chains(ctx);
  if (st) return st;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
  dqmc_sweep_stats S{};
  double prec_sum = 0.0, sign_sum = 0.0;
  int64_t events = 0;
  int err = 0;
  for (const ChainDev& C : ctx->chains_h) {
    S.proposals += C.proposals;
    S.accepted += C.accepted;
    for (int s = 0; s < C.nfl; ++s) {
      prec_sum += C.prec_sum[s];
      S.prec_green_max = std::max(S.prec_green_max, C.prec_max[s]);
    }
    events += C.prec_events;
    S.prec_phase_max = std::max(S.prec_phase_max, C.phase_max);
    sign_sum += C.sweep_sign_sum;
    err |= C.error;
  }
  // per-phase times of the slowest chain (the critical path of the launch)
  {
    int dev = 0, khz = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
    const double per_ms = khz > 0 ? (double)khz : 1.0;
    double best = -1.0;
    for (const ChainDev& C : ctx->chains_h)
      for (int s = 0; s < C.nfl; ++s) {
        const double tot = (double)(C.cyc[s][0] + C.cyc[s][1] + C.cyc[s][2] + C.cyc[s][3]);
        if (tot > best) {
          best = tot;
          S.ms_update = (float)(C.cyc[s][0] / per_ms);
          S.ms_wrap = (float)(C.cyc[s][1] / per_ms);
          S.ms_stab = (float)(C.cyc[s][2] / per_ms);
          S.ms_measure = (float)(C.cyc[s][3] / per_ms);
          for (int q = 0; q < 8; ++q) S.ms_detail[q] = (float)(C.cycd[s][q] / per_ms);
        }
      }
  }
  S.prec_green_mean = events ? prec_sum / (double)events : 0.0;
  S.mean_sign = n_sweeps ? sign_sum / ((double)n_sweeps * n) : 0.0;
  S.ms_total = ms;
  *stats = S;
  if (err & 2) {
    for (const ChainDev& C : ctx->chains_h)
      if (C.error & 2) return timeout_message(ctx, C);
  }
  if (err) return fail(ctx, DQMC_EUNSTABLE, "singular matrix in the stabilisation");
  if (ctx->opts.unstable_threshold > 0.0 && S.prec_green_max > ctx->opts.unstable_threshold)
    return fail(ctx, DQMC_EUNSTABLE, "max|G_wrap - G_fresh| = %.3e exceeds %.3e", S.prec_green_max,
                ctx->opts.unstable_threshold);
  return DQMC_OK;
}

dqmc_status dqmc_greens(dqmc_ctx* ctx, int32_t chain, int32_t flavor, int32_t fresh, double* out,
                        int32_t out_is_device, double* logdet_out, int32_t* sign_out) {
  if (!ctx) return DQMC_EINVAL;
  if (chain < 0 || chain >= (int)ctx->chains_h.size() || flavor < 0 || flavor >= ctx->nfl || !out)
    return fail(ctx, DQMC_EINVAL, "chain or flavor out of range, or null output");
  const int N = ctx->chains_h[chain].N;
  double* src;
  if (fresh) {
    dqmc::set_smem_bytes(ctx->smem);
    CUDA_TRY(ctx, dqmc::launch_fresh_green(ctx->chains_d, (int)ctx->chains_h.size(), ctx->nfl, ctx->opts.precision, 0,
                                           ctx->scratch, chain, ctx->stream));
    src = ctx->scratch + (size_t)flavor * N * N;
  } else {
    CUDA_TRY(ctx, dqmc::launch_copy_green(ctx->chains_d, chain, flavor, ctx->kprec, ctx->scratch, ctx->stream));
    src = ctx->scratch;
  }
  CUDA_TRY(ctx, cudaMemcpyAsync(out, src, sizeof(double) * N * N,
                                out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
  dqmc_status st = download_chains(ctx);
  if (st) return st;
  const ChainDev& C = ctx->chains_h[chain];
  if (C.error) return fail(ctx, DQMC_EUNSTABLE, "singular matrix in the stabilisation");
  if (logdet_out) *logdet_out = C.logdet[flavor];
  if (sign_out) *sign_out = C.fresh_sign[flavor];
  return DQMC_OK;
}

dqmc_status dqmc_greens_tau(dqmc_ctx* ctx, int32_t chain, int32_t flavor, int32_t tau, double* out,
                            int32_t out_is_device) {
  if (!ctx) return DQMC_EINVAL;
  if (chain < 0 || chain >= (int)ctx->chains_h.size() || flavor < 0 || flavor >= ctx->nfl || !out)
    return fail(ctx, DQMC_EINVAL, "chain or flavor out of range, or null output");
  const ChainDev& H = ctx->chains_h[chain];
  if (tau < 0 || tau > H.L) return fail(ctx, DQMC_EINVAL, "tau must be in [0, %d]", H.L);
  const int N = H.N;
  dqmc::set_smem_bytes(ctx->smem);
  CUDA_TRY(ctx, dqmc::launch_green_tau(ctx->chains_d, chain, ctx->nfl, ctx->opts.precision, tau, ctx->scratch,
                                       ctx->stream));
  CUDA_TRY(ctx, cudaMemcpyAsync(out, ctx->scratch + (size_t)flavor * N * N, sizeof(double) * N * N,
                                out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
  dqmc_status st = download_chains(ctx);
  if (st) return st;
  if (ctx->chains_h[chain].error) return fail(ctx, DQMC_EUNSTABLE, "singular matrix in the stabilisation");
  return DQMC_OK;
}

dqmc_status dqmc_measure(dqmc_ctx* ctx, double* out, double* sign_sum, int64_t* n_meas) {
  if (!ctx) return DQMC_EINVAL;
  if (!out || !sign_sum || !n_meas) return fail(ctx, DQMC_EINVAL, "null output");
  dqmc_status st = download_chains(ctx);
  if (st) return st;
  for (size_t c = 0; c < ctx->chains_h.size(); ++c) {
    const ChainDev& C = ctx->chains_h[c];
    for (int q = 0; q < 4; ++q) out[c * 4 + q] = C.meas[q];
    sign_sum[c] = C.meas_sign;
    n_meas[c] = C.n_meas;
  }
  return DQMC_OK;
}

}  // extern "C"

namespace {

// Pair classes per model as CSR lists (pairs x * N + y sorted by class, then
// by x, y) and the per-chain offsets into them; rejects classes outside
// [-1, n_class).
struct ClassLists {
  std::vector<int> csr, pairs, ccsr, cpairs, cncls;
  int max_cls = 0;
};

dqmc_status build_class_lists(dqmc_ctx* ctx, const int32_t* pair_class, const int32_t* n_class, ClassLists& L) {
  const int nm = (int)ctx->models.size(), nch = (int)ctx->chains_h.size();
  std::vector<int> mcsr(nm), mpairs(nm);
  size_t coff = 0;
  for (int m = 0; m < nm; ++m) {
    const int N = ctx->models[m].d.n_sites, nc = n_class[m];
    if (nc < 1) return fail(ctx, DQMC_EINVAL, "model %d: n_class < 1", m);
    L.max_cls = nc > L.max_cls ? nc : L.max_cls;
    const int32_t* cl = pair_class + coff;
    std::vector<int> cnt(nc + 1, 0);
    for (int e = 0; e < N * N; ++e) {
      if (cl[e] < -1 || cl[e] >= nc) return fail(ctx, DQMC_EINVAL, "model %d: pair class %d out of range", m, cl[e]);
      if (cl[e] >= 0) ++cnt[cl[e] + 1];
    }
    for (int k = 0; k < nc; ++k) cnt[k + 1] += cnt[k];
    mcsr[m] = (int)L.csr.size();
    mpairs[m] = (int)L.pairs.size();
    L.csr.insert(L.csr.end(), cnt.begin(), cnt.end());
    std::vector<int> fill(cnt.begin(), cnt.end() - 1);
    L.pairs.resize(L.pairs.size() + cnt[nc]);
    for (int e = 0; e < N * N; ++e)
      if (cl[e] >= 0) L.pairs[mpairs[m] + fill[cl[e]]++] = e;
    coff += (size_t)N * N;
  }
  L.ccsr.resize(nch);
  L.cpairs.resize(nch);
  L.cncls.resize(nch);
  for (int c = 0; c < nch; ++c) {
    const int m = ctx->chain_model[c];
    L.ccsr[c] = mcsr[m];
    L.cpairs[c] = mpairs[m];
    L.cncls[c] = n_class[m];
  }
  if (L.pairs.empty()) L.pairs.push_back(0);
  return DQMC_OK;
}

// Device copy of the class lists: one int buffer [csr | pairs | ccsr | cpairs | cncls].
struct ClassListsDev {
  int* buf = nullptr;
  const int *csr = nullptr, *pairs = nullptr, *ccsr = nullptr, *cpairs = nullptr, *cncls = nullptr;
  ~ClassListsDev() { cudaFree(buf); }
};

dqmc_status upload_class_lists(dqmc_ctx* ctx, const ClassLists& L, ClassListsDev& D) {
  const size_t nch = L.ccsr.size();
  const size_t n = L.csr.size() + L.pairs.size() + 3 * nch;
  if (cudaMalloc((void**)&D.buf, sizeof(int) * n) != cudaSuccess) {
    D.buf = nullptr;
    cudaGetLastError();
    return fail(ctx, DQMC_ENOMEM, "no device memory for the pair classes");
  }
  std::vector<int> h;
  h.reserve(n);
  h.insert(h.end(), L.csr.begin(), L.csr.end());
  h.insert(h.end(), L.pairs.begin(), L.pairs.end());
  h.insert(h.end(), L.ccsr.begin(), L.ccsr.end());
  h.insert(h.end(), L.cpairs.begin(), L.cpairs.end());
  h.insert(h.end(), L.cncls.begin(), L.cncls.end());
  CUDA_TRY(ctx, cudaMemcpyAsync(D.buf, h.data(), sizeof(int) * n, cudaMemcpyHostToDevice, ctx->stream));
  D.csr = D.buf;
  D.pairs = D.csr + L.csr.size();
  D.ccsr = D.pairs + L.pairs.size();
  D.cpairs = D.ccsr + nch;
  D.cncls = D.cpairs + nch;
  return DQMC_OK;
}

// The time-displaced measurement shared by dqmc_measure_tau (sums) and
// dqmc_measure_tau_corr (class-resolved correlations, tc.part set).
dqmc_status run_tau_measure(dqmc_ctx* ctx, int32_t n_tau, const double* site_phase, double* out, int32_t* sign,
                            double* prec, const dqmc::TauCorrArgs& tc) {
  int maxL = 0;
  for (const ChainDev& C : ctx->chains_h) maxL = C.L > maxL ? C.L : maxL;
  if (n_tau < 0 || n_tau > maxL) return fail(ctx, DQMC_EINVAL, "n_tau outside 0..%d", maxL);
  const int nch = (int)ctx->chains_h.size(), nfl = ctx->nfl, pld = ctx->maxN;
  std::vector<size_t> moff(ctx->models.size() + 1, 0);
  for (size_t m = 0; m < ctx->models.size(); ++m) moff[m + 1] = moff[m] + ctx->models[m].d.n_sites;
  std::vector<double> ph((size_t)nch * pld, 0.0);
  for (int c = 0; c < nch; ++c) {
    const int m = ctx->chain_model[c];
    for (int x = 0; x < ctx->chains_h[c].N; ++x) {
      const double v = site_phase ? site_phase[moff[m] + x] : 1.0;
      if (!std::isfinite(v)) return fail(ctx, DQMC_EINVAL, "non-finite site phase");
      ph[(size_t)c * pld + x] = v;
    }
  }
  const size_t tw_stride = (size_t)4 * ctx->maxN * ctx->maxld;
  if (!ctx->tau_work) {
    if (cudaMalloc((void**)&ctx->tau_work, sizeof(double) * tw_stride * nch * nfl) != cudaSuccess) {
      ctx->tau_work = nullptr;
      cudaGetLastError();
      return fail(ctx, DQMC_ENOMEM, "no device memory for the time-displaced workspace");
    }
  }
  const size_t nobs = (size_t)nch * (n_tau + 1) * nfl * 3;
  double *ph_d = nullptr, *obs_d = nullptr, *prec_d = nullptr;
  int* sg_d = nullptr;
  dqmc_status st = DQMC_OK;
  auto cleanup = [&]() {
    cudaFree(ph_d);
    cudaFree(obs_d);
    cudaFree(prec_d);
    cudaFree(sg_d);
  };
  if (cudaMalloc((void**)&ph_d, sizeof(double) * ph.size()) != cudaSuccess ||
      cudaMalloc((void**)&obs_d, sizeof(double) * nobs) != cudaSuccess ||
      cudaMalloc((void**)&prec_d, sizeof(double) * nch * nfl * 3) != cudaSuccess ||
      cudaMalloc((void**)&sg_d, sizeof(int) * nch * nfl) != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    return fail(ctx, DQMC_ENOMEM, "no device memory for the time-displaced outputs");
  }
  std::vector<double> prec_h((size_t)nch * nfl * 3);
  do {
    if (cudaMemcpyAsync(ph_d, ph.data(), sizeof(double) * ph.size(), cudaMemcpyHostToDevice, ctx->stream) !=
        cudaSuccess) { st = fail(ctx, DQMC_ECUDA, "phase upload failed"); break; }
    dqmc::set_smem_bytes(ctx->smem);
    cudaError_t e = dqmc::launch_tau_measure(ctx->chains_d, nch, nfl, n_tau, ph_d, pld, ctx->tau_work, tw_stride,
                                             obs_d, prec_d, sg_d, tc, ctx->stream);
    if (e != cudaSuccess) { st = fail(ctx, DQMC_ECUDA, "tau measurement launch: %s", cudaGetErrorString(e)); break; }
    if ((out && cudaMemcpyAsync(out, obs_d, sizeof(double) * nobs, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess) ||
        cudaMemcpyAsync(sign, sg_d, sizeof(int) * nch * nfl, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
        cudaMemcpyAsync(prec_h.data(), prec_d, sizeof(double) * prec_h.size(), cudaMemcpyDeviceToHost,
                        ctx->stream) != cudaSuccess) { st = fail(ctx, DQMC_ECUDA, "download failed"); break; }
    st = download_chains(ctx);
    if (st) break;
    for (const ChainDev& C : ctx->chains_h)
      if (C.error) { st = fail(ctx, DQMC_EUNSTABLE, "chain %u: singular matrix in the stabilisation", C.chain_id); break; }
  } while (false);
  cleanup();
  if (st) return st;
  if (prec) {
    double sum = 0.0, mx = 0.0, ev = 0.0;
    for (size_t q = 0; q < prec_h.size(); q += 3) {
      sum += prec_h[q];
      mx = prec_h[q + 1] > mx ? prec_h[q + 1] : mx;
      ev += prec_h[q + 2];
    }
    prec[0] = ev > 0 ? sum / ev : 0.0;
    prec[1] = mx;
  }
  return DQMC_OK;
}

}  // namespace

extern "C" {

dqmc_status dqmc_measure_tau(dqmc_ctx* ctx, int32_t n_tau, const double* site_phase, double* out, int32_t* sign,
                             double* prec) {
  if (!ctx) return DQMC_EINVAL;
  if (!out || !sign) return fail(ctx, DQMC_EINVAL, "null output");
  return run_tau_measure(ctx, n_tau, site_phase, out, sign, prec, dqmc::TauCorrArgs{});
}

dqmc_status dqmc_measure_tau_corr(dqmc_ctx* ctx, int32_t n_tau, const int32_t* pair_class, const int32_t* n_class,
                                  double* out, int32_t* sign) {
  if (!ctx) return DQMC_EINVAL;
  if (!pair_class || !n_class || !out || !sign) return fail(ctx, DQMC_EINVAL, "null argument");
  if (ctx->nfl != 2) return fail(ctx, DQMC_EINVAL, "correlation functions need the two flavors of the spin-z decoupling");
  int maxL = 0;
  for (const ChainDev& C : ctx->chains_h) maxL = C.L > maxL ? C.L : maxL;
  if (n_tau < 0 || n_tau > maxL) return fail(ctx, DQMC_EINVAL, "n_tau outside 0..%d", maxL);
  ClassLists L;
  dqmc_status st = build_class_lists(ctx, pair_class, n_class, L);
  if (st) return st;
  ClassListsDev D;
  if ((st = upload_class_lists(ctx, L, D))) return st;
  const int nch = (int)ctx->chains_h.size();
  const size_t npart = (size_t)nch * (n_tau + 1) * 2 * L.max_cls * 2;
  const size_t ndens = (size_t)nch * (n_tau + 1) * 2 * ctx->maxN;
  const size_t nout = (size_t)nch * (n_tau + 1) * L.max_cls * 3;
  double* work = nullptr;
  if (cudaMalloc((void**)&work, sizeof(double) * (npart + ndens + nout)) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, DQMC_ENOMEM, "no device memory for the time-displaced correlations");
  }
  dqmc::TauCorrArgs tc;
  tc.csr_all = D.csr;
  tc.pairs_all = D.pairs;
  tc.chain_csr = D.ccsr;
  tc.chain_pairs = D.cpairs;
  tc.chain_ncls = D.cncls;
  tc.max_cls = L.max_cls;
  tc.part = work;
  tc.dens = work + npart;
  tc.dens_ld = ctx->maxN;
  double* out_d = work + npart + ndens;
  std::vector<int32_t> sg2((size_t)nch * 2);
  st = run_tau_measure(ctx, n_tau, nullptr, nullptr, sg2.data(), nullptr, tc);
  if (!st) {
    cudaError_t e = dqmc::launch_tau_corr_combine(ctx->chains_d, nch, n_tau, tc, out_d, ctx->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(out, out_d, sizeof(double) * nout, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) st = fail(ctx, DQMC_ECUDA, "time-displaced correlations: %s", cudaGetErrorString(e));
  }
  cudaFree(work);
  if (st) return st;
  for (int c = 0; c < nch; ++c) sign[c] = sg2[2 * c] * sg2[2 * c + 1];
  return DQMC_OK;
}

dqmc_status dqmc_measure_corr(dqmc_ctx* ctx, const int32_t* pair_class, const int32_t* n_class, double* out,
                              int32_t* sign) {
  if (!ctx) return DQMC_EINVAL;
  if (!pair_class || !n_class || !out || !sign) return fail(ctx, DQMC_EINVAL, "null argument");
  if (ctx->nfl != 2) return fail(ctx, DQMC_EINVAL, "correlation functions need the two flavors of the spin-z decoupling");
  const int nch = (int)ctx->chains_h.size();
  ClassLists L;
  dqmc_status st = build_class_lists(ctx, pair_class, n_class, L);
  if (st) return st;
  ClassListsDev D;
  if ((st = upload_class_lists(ctx, L, D))) return st;
  double* out_d = nullptr;
  const size_t nout = (size_t)nch * L.max_cls * 4;
  if (cudaMalloc((void**)&out_d, sizeof(double) * nout) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, DQMC_ENOMEM, "no device memory for the correlation functions");
  }
  do {
    cudaError_t e = dqmc::launch_corr(ctx->chains_d, nch, ctx->kprec, D.csr, D.pairs, D.ccsr, D.cpairs, D.cncls,
                                      L.max_cls, out_d, ctx->stream);
    if (e != cudaSuccess) { st = fail(ctx, DQMC_ECUDA, "correlation launch: %s", cudaGetErrorString(e)); break; }
    if (cudaMemcpyAsync(out, out_d, sizeof(double) * nout, cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess) {
      st = fail(ctx, DQMC_ECUDA, "download failed");
      break;
    }
    st = download_chains(ctx);
  } while (false);
  cudaFree(out_d);
  if (st) return st;
  for (int c = 0; c < nch; ++c) sign[c] = ctx->chains_h[c].sign;
  return DQMC_OK;
}

dqmc_status dqmc_get_fields(dqmc_ctx* ctx, int8_t* out, uint64_t* rng_counter) {
  if (!ctx) return DQMC_EINVAL;
  if (!out) return fail(ctx, DQMC_EINVAL, "null output");
  size_t off = 0;
  for (const ChainDev& C : ctx->chains_h) {
    const size_t nf = (size_t)C.L * C.MV;
    CUDA_TRY(ctx, cudaMemcpyAsync(out + off, C.fields, nf, cudaMemcpyDeviceToHost, ctx->stream));
    off += nf;
  }
  if (rng_counter) *rng_counter = ctx->sweep_counter;
  return sync_check(ctx);
}

dqmc_status dqmc_set_fields(dqmc_ctx* ctx, const int8_t* in, uint64_t rng_counter) {
  if (!ctx) return DQMC_EINVAL;
  if (!in) return fail(ctx, DQMC_EINVAL, "null input");
  // every chain is checked before any is replaced: a rejected call leaves the ensemble as it was
  size_t off = 0;
  for (const ChainDev& C : ctx->chains_h) {
    const size_t nf = (size_t)C.L * C.MV;
    for (size_t q = 0; q < nf; ++q) {
      const int8_t f = in[off + q];
      const bool ok = (C.ft == DQMC_FIELD_ISING) ? (f == 1 || f == -1) : (f == 1 || f == -1 || f == 2 || f == -2);
      if (!ok) return fail(ctx, DQMC_EINVAL, "chain %u: invalid field value %d", C.chain_id, (int)f);
    }
    off += nf;
  }
  off = 0;
  for (const ChainDev& C : ctx->chains_h) {
    const size_t nf = (size_t)C.L * C.MV;
    CUDA_TRY(ctx, cudaMemcpyAsync(C.fields, in + off, nf, cudaMemcpyHostToDevice, ctx->stream));
    off += nf;
  }
  ctx->sweep_counter = rng_counter;
  return initial_fill(ctx);
}

dqmc_status dqmc_logdet_backward(dqmc_ctx* ctx, int32_t model_index, const int8_t* fields, int32_t n_cfg,
                                 double* logdet, double* grad_K, double* grad_U) {
  if (!ctx) return DQMC_EINVAL;
  if (model_index < 0 || model_index >= (int)ctx->models.size() || !fields || n_cfg < 1 || !logdet || !grad_K ||
      !grad_U)
    return fail(ctx, DQMC_EINVAL, "bad model index, empty configuration list or null output");
  const ModelHost& M = ctx->models[model_index];
  const int N = M.d.n_sites, nfl = M.d.n_flavors, MV = M.d.n_vertices, L = M.d.L;
  for (size_t q = 0; q < (size_t)n_cfg * L * MV; ++q) {
    const int8_t f = fields[q];
    const bool ok = (M.d.field_type == DQMC_FIELD_ISING) ? (f == 1 || f == -1) : (f == 1 || f == -1 || f == 2 || f == -2);
    if (!ok) return fail(ctx, DQMC_EINVAL, "invalid field value %d", (int)f);
  }
  const size_t per = chain_layout(M, DQMC_PREC_FP64, 1, nullptr, nullptr);
  unsigned char* arena = nullptr;
  if (cudaMalloc((void**)&arena, per * n_cfg) != cudaSuccess)
    return fail(ctx, DQMC_ENOMEM, "gradient workspace of %zu bytes", per * n_cfg);
  std::vector<ChainDev> ch(n_cfg, ChainDev{});
  for (int c = 0; c < n_cfg; ++c) {
    chain_layout(M, DQMC_PREC_FP64, 1, arena + per * c, &ch[c]);
    fill_model_fields(M, ch[c]);
    ch[c].chain_id = (uint32_t)c;
    ch[c].sign = 1;
  }
  ChainDev* ch_d = nullptr;
  double *V_d = nullptr, *w_d = nullptr, *gK_d = nullptr, *gU_d = nullptr;
  std::vector<double> Vh((size_t)nfl * N * N), wh((size_t)nfl * N);
  for (int s = 0; s < nfl; ++s) {
    std::copy(M.eigvec[s].begin(), M.eigvec[s].end(), Vh.begin() + (size_t)s * N * N);
    std::copy(M.eigval[s].begin(), M.eigval[s].end(), wh.begin() + (size_t)s * N);
  }
  dqmc_status st = DQMC_OK;
  auto cleanup = [&]() {
    cudaFree(arena);
    cudaFree(ch_d);
    cudaFree(V_d);
    cudaFree(w_d);
    cudaFree(gK_d);
    cudaFree(gU_d);
  };
#define GRAD_TRY(expr)                                                                 \
  do {                                                                                 \
    cudaError_t e_ = (expr);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      st = fail(ctx, DQMC_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_));             \
      cleanup();                                                                       \
      return st;                                                                       \
    }                                                                                  \
  } while (0)
  GRAD_TRY(cudaMemsetAsync(arena, 0, per * n_cfg, ctx->stream));
  for (int c = 0; c < n_cfg; ++c)
    GRAD_TRY(cudaMemcpyAsync(ch[c].fields, fields + (size_t)c * L * MV, (size_t)L * MV, cudaMemcpyHostToDevice,
                             ctx->stream));
  GRAD_TRY(cudaMalloc((void**)&ch_d, sizeof(ChainDev) * n_cfg));
  GRAD_TRY(cudaMemcpyAsync(ch_d, ch.data(), sizeof(ChainDev) * n_cfg, cudaMemcpyHostToDevice, ctx->stream));
  GRAD_TRY(cudaMalloc((void**)&V_d, sizeof(double) * Vh.size()));
  GRAD_TRY(cudaMalloc((void**)&w_d, sizeof(double) * wh.size()));
  GRAD_TRY(cudaMalloc((void**)&gK_d, sizeof(double) * (size_t)n_cfg * nfl * N * N));
  GRAD_TRY(cudaMalloc((void**)&gU_d, sizeof(double) * (size_t)n_cfg * nfl));
  GRAD_TRY(cudaMemcpyAsync(V_d, Vh.data(), sizeof(double) * Vh.size(), cudaMemcpyHostToDevice, ctx->stream));
  GRAD_TRY(cudaMemcpyAsync(w_d, wh.data(), sizeof(double) * wh.size(), cudaMemcpyHostToDevice, ctx->stream));
  dqmc::set_smem_bytes(dqmc::sweep_smem_bytes(N, M.ld, MV, 1, 0));
  GRAD_TRY(dqmc::launch_logdet_grad(ch_d, n_cfg, nfl, V_d, w_d, gK_d, gU_d, nullptr, ctx->stream));
  GRAD_TRY(cudaMemcpyAsync(grad_K, gK_d, sizeof(double) * (size_t)n_cfg * nfl * N * N, cudaMemcpyDeviceToHost,
                           ctx->stream));
  GRAD_TRY(cudaMemcpyAsync(grad_U, gU_d, sizeof(double) * (size_t)n_cfg * nfl, cudaMemcpyDeviceToHost, ctx->stream));
  GRAD_TRY(cudaMemcpyAsync(ch.data(), ch_d, sizeof(ChainDev) * n_cfg, cudaMemcpyDeviceToHost, ctx->stream));
  GRAD_TRY(cudaStreamSynchronize(ctx->stream));
#undef GRAD_TRY
  for (int c = 0; c < n_cfg; ++c) {
    if (ch[c].error) st = fail(ctx, DQMC_EUNSTABLE, "configuration %d: singular matrix in the stabilisation", c);
    for (int s = 0; s < nfl; ++s) logdet[(size_t)c * nfl + s] = ch[c].logdet[s];
  }
  cleanup();
  return st;
}

dqmc_status dqmc_energy_backward(dqmc_ctx* ctx, int32_t model_index, const int8_t* fields, int32_t n_cfg,
                                 double* energy, double* grad_K, double* grad_U) {
  if (!ctx) return DQMC_EINVAL;
  if (model_index < 0 || model_index >= (int)ctx->models.size() || !fields || n_cfg < 1 || !energy || !grad_K ||
      !grad_U)
    return fail(ctx, DQMC_EINVAL, "bad model index, empty configuration list or null output");
  const ModelHost& M = ctx->models[model_index];
  const int N = M.d.n_sites, nfl = M.d.n_flavors, MV = M.d.n_vertices, L = M.d.L, ld = M.ld;
  for (size_t q = 0; q < (size_t)n_cfg * L * MV; ++q) {
    const int8_t f = fields[q];
    const bool ok = (M.d.field_type == DQMC_FIELD_ISING) ? (f == 1 || f == -1) : (f == 1 || f == -1 || f == 2 || f == -2);
    if (!ok) return fail(ctx, DQMC_EINVAL, "invalid field value %d", (int)f);
  }
  const size_t per = chain_layout(M, DQMC_PREC_FP64, 1, nullptr, nullptr);
  const size_t mat = (size_t)N * ld;
  std::vector<ChainDev> ch(n_cfg, ChainDev{});
  unsigned char* arena = nullptr;
  ChainDev* ch_d = nullptr;
  double *V_d = nullptr, *w_d = nullptr, *G0_d = nullptr, *ew_d = nullptr, *gK_d = nullptr, *gU_d = nullptr,
         *ep_d = nullptr;
  dqmc_status st = DQMC_OK;
  auto cleanup = [&]() {
    cudaFree(arena);
    cudaFree(ch_d);
    cudaFree(V_d);
    cudaFree(w_d);
    cudaFree(G0_d);
    cudaFree(ew_d);
    cudaFree(gK_d);
    cudaFree(gU_d);
    cudaFree(ep_d);
  };
#define EGRAD_TRY(expr)                                                                \
  do {                                                                                 \
    cudaError_t e_ = (expr);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      st = fail(ctx, DQMC_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_));             \
      cleanup();                                                                       \
      return st;                                                                       \
    }                                                                                  \
  } while (0)
  EGRAD_TRY(cudaMalloc((void**)&arena, per * n_cfg));
  EGRAD_TRY(cudaMemsetAsync(arena, 0, per * n_cfg, ctx->stream));
  for (int c = 0; c < n_cfg; ++c) {
    chain_layout(M, DQMC_PREC_FP64, 1, arena + per * c, &ch[c]);
    fill_model_fields(M, ch[c]);
    ch[c].chain_id = (uint32_t)c;
    ch[c].sign = 1;
    EGRAD_TRY(cudaMemcpyAsync(ch[c].fields, fields + (size_t)c * L * MV, (size_t)L * MV, cudaMemcpyHostToDevice,
                              ctx->stream));
  }
  std::vector<double> Vh((size_t)nfl * N * N), wh((size_t)nfl * N);
  for (int s = 0; s < nfl; ++s) {
    std::copy(M.eigvec[s].begin(), M.eigvec[s].end(), Vh.begin() + (size_t)s * N * N);
    std::copy(M.eigval[s].begin(), M.eigval[s].end(), wh.begin() + (size_t)s * N);
  }
  EGRAD_TRY(cudaMalloc((void**)&ch_d, sizeof(ChainDev) * n_cfg));
  EGRAD_TRY(cudaMemcpyAsync(ch_d, ch.data(), sizeof(ChainDev) * n_cfg, cudaMemcpyHostToDevice, ctx->stream));
  EGRAD_TRY(cudaMalloc((void**)&V_d, sizeof(double) * Vh.size()));
  EGRAD_TRY(cudaMalloc((void**)&w_d, sizeof(double) * wh.size()));
  EGRAD_TRY(cudaMemcpyAsync(V_d, Vh.data(), sizeof(double) * Vh.size(), cudaMemcpyHostToDevice, ctx->stream));
  EGRAD_TRY(cudaMemcpyAsync(w_d, wh.data(), sizeof(double) * wh.size(), cudaMemcpyHostToDevice, ctx->stream));
  EGRAD_TRY(cudaMalloc((void**)&G0_d, sizeof(double) * (size_t)n_cfg * nfl * N * N));
  EGRAD_TRY(cudaMalloc((void**)&ew_d, sizeof(double) * (size_t)n_cfg * nfl * 6 * mat));
  EGRAD_TRY(cudaMalloc((void**)&gK_d, sizeof(double) * (size_t)n_cfg * nfl * N * N));
  EGRAD_TRY(cudaMalloc((void**)&gU_d, sizeof(double) * (size_t)n_cfg * nfl));
  EGRAD_TRY(cudaMalloc((void**)&ep_d, sizeof(double) * (size_t)n_cfg * nfl * 3));
  dqmc::set_smem_bytes(dqmc::sweep_smem_bytes(N, ld, MV, 1, 0));
  EGRAD_TRY(dqmc::launch_energy_grad(ch_d, n_cfg, nfl, V_d, w_d, G0_d, ew_d, gK_d, gU_d, ep_d, ctx->stream));
  std::vector<double> gU((size_t)n_cfg * nfl), ep((size_t)n_cfg * nfl * 3);
  EGRAD_TRY(cudaMemcpyAsync(grad_K, gK_d, sizeof(double) * (size_t)n_cfg * nfl * N * N, cudaMemcpyDeviceToHost,
                            ctx->stream));
  EGRAD_TRY(cudaMemcpyAsync(gU.data(), gU_d, sizeof(double) * gU.size(), cudaMemcpyDeviceToHost, ctx->stream));
  EGRAD_TRY(cudaMemcpyAsync(ep.data(), ep_d, sizeof(double) * ep.size(), cudaMemcpyDeviceToHost, ctx->stream));
  EGRAD_TRY(cudaMemcpyAsync(ch.data(), ch_d, sizeof(ChainDev) * n_cfg, cudaMemcpyDeviceToHost, ctx->stream));
  EGRAD_TRY(cudaStreamSynchronize(ctx->stream));
#undef EGRAD_TRY
  for (int c = 0; c < n_cfg; ++c) {
    if (ch[c].error) st = fail(ctx, DQMC_EUNSTABLE, "configuration %d: singular matrix in the stabilisation", c);
    double kin = 0.0, part = 0.0, pot = 0.0, gu = 0.0;
    for (int s = 0; s < nfl; ++s) {
      kin += ep[((size_t)c * nfl + s) * 3 + 0];
      part += ep[((size_t)c * nfl + s) * 3 + 1];
      pot += ep[((size_t)c * nfl + s) * 3 + 2];
      gu += gU[(size_t)c * nfl + s];
    }
    energy[(size_t)c * 4 + 0] = kin;
    energy[(size_t)c * 4 + 1] = pot;
    energy[(size_t)c * 4 + 2] = part;
    energy[(size_t)c * 4 + 3] = kin + pot;
    grad_U[c] = gu;
  }
  cleanup();
  return st;
}

const char* dqmc_last_error(const dqmc_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

void dqmc_destroy(dqmc_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  cudaFree(ctx->arena);
  cudaFree(ctx->chains_d);
  cudaFree(ctx->order_d);
  cudaFree(ctx->scratch);
  cudaFree(ctx->tau_work);
  for (void* p : ctx->model_allocs) cudaFree(p);
  if (ctx->ev0) cudaEventDestroy(ctx->ev0);
  if (ctx->ev1) cudaEventDestroy(ctx->ev1);
  delete ctx;
}

}  // extern "C"
