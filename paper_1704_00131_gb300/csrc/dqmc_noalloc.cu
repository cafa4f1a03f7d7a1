// Allocation-free entry point (see the section comment below); its scratch array
// lives in this translation unit only.
#include "dqmc_device.cuh"

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
  Smem S = carve_smem(smem_raw, ld, C.MV);
  // the vertex sites are caller device data the host cannot inspect: they must
  // be distinct and in [0, N) (they index the slice potential in shared memory);
  // otherwise the call returns sign 0, log|det| 0 and a G of NaNs
  for (int x = threadIdx.x; x < N; x += kThreads) S.qinv[x] = 0;
  __syncthreads();
  int bad_site = 0;
  for (int k = threadIdx.x; k < C.MV; k += kThreads) {
    const int site = C.site[k];
    if (site < 0 || site >= N) bad_site = 1;
    else if (atomicAdd(&S.qinv[site], 1) != 0) bad_site = 1;
  }
  if (__syncthreads_or(bad_site)) {
    for (int e = threadIdx.x; e < N * N; e += kThreads) out[(size_t)s * N * N + e] = __longlong_as_double(0x7ff8000000000000LL);
    if (threadIdx.x == 0) {
      if (logdet_out) logdet_out[s] = 0.0;
      if (sign_out) sign_out[s] = 0;
    }
    return;
  }
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
