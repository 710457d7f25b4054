// pdhg_kkt_noalloc: the KKT evaluation without any memory allocation.
//
// Some callers cannot let a library allocate: applications whose device
// memory is owned by their own pool or framework allocator (a cudaMalloc
// behind its back can fail or fragment a budget it has fully committed),
// services with a fixed memory budget per process, and code on a latency-
// critical path where cudaMalloc/cudaFree would synchronize the device. This
// entry point serves them: it computes the same KKT measures as pdhg_kkt, for
// a point (x, y) the caller supplies, of an LP the caller keeps on the device
// as two CSR matrices (A and A^T). It allocates nothing on the device or the
// host: the only scratch, the per-block partial sums of the reductions, lives
// in the file-scope array below, which every GPU that loads this library holds
// (KKT_NA_SCRATCH_DOUBLES doubles, 96 KiB) until the process exits.
//
// Limits and sharing rules:
//   - at most KKT_NA_MAX_BLOCKS blocks per pass (the scratch holds one row of
//     partial sums per block); larger requests are rejected with
//     PDHG_ERR_INVALID;
//   - every call on a device uses the same array and leaves its contents
//     behind; each call overwrites every slot it reads before reading it, so
//     nothing has to start at zero;
//   - calls whose kernels overlap on the same GPU (different streams or
//     threads without ordering between them) race on the array and give
//     wrong results: order them on one stream or serialize them.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "../../include/pdhg.h"
#include "common.cuh"

namespace {

constexpr int KKT_NA_MAX_BLOCKS = 1024;
constexpr int KKT_NA_Q = 12;  // quantities per block (10 used)
constexpr int KKT_NA_SCRATCH_DOUBLES = KKT_NA_MAX_BLOCKS * KKT_NA_Q;
constexpr int KKT_NA_TPB = 256;
constexpr int KKT_NA_MAX_DEVICES = 64;

// partial sums [block][q], then the KKT_NA_Q final sums
static __device__ __align__(256) double g_kkt_scratch[KKT_NA_SCRATCH_DOUBLES + KKT_NA_Q];

enum {
  NA_RD2 = 0,  // sum max(0, A^T y - c)^2
  NA_RDINF,    // max of the same
  NA_CX,       // c^T x
  NA_XZ,       // x^T z, z = max(0, c - A^T y)
  NA_C2,       // ||c||^2
  NA_RP2,      // sum (b - A x)^2
  NA_RPINF,    // max |b - A x|
  NA_BY,       // b^T y
  NA_B2,       // ||b||^2
  NA_COUNT
};

#ifdef PDHG_CHECKED
// checked build: set when a column index of the caller's CSR lies outside the
// vector it indexes (that entry is then skipped); read and cleared by the
// finalizing kernel of the same call
static __device__ unsigned g_na_check;
#endif

// device address of g_kkt_scratch per device (host code cannot use the
// symbol's name as an address)
double* g_scratch_ptr[KKT_NA_MAX_DEVICES] = {};
std::mutex g_scratch_mu;

__device__ __forceinline__ double na_relu(double v) { return v < 0.0 ? 0.0 : v; }

// one warp per row, lane-strided dot product; result in lane 0. A warp per
// row suits small LPs and LPs with evenly filled rows; a row of thousands of
// entries is reduced by one warp alone (the engine's own evaluation splits
// such rows over panels instead).
__device__ __forceinline__ double na_row_dot(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                             const double* __restrict__ v, const double* __restrict__ vec,
                                             long long row, int lane, long long veclen) {
  const long long beg = rp[row], end = rp[row + 1];
  double acc = 0.0;
  for (long long k = beg + lane; k < end; k += 32) {
    const int c = ci[k];
#ifdef PDHG_CHECKED
    if ((unsigned long long)(unsigned)c >= (unsigned long long)veclen) {
      atomicOr(&g_na_check, 1u);
      continue;
    }
#else
    (void)veclen;
#endif
    acc += v[k] * vec[c];
  }
  return pdhg::warp_sum(acc);
}

__global__ void __launch_bounds__(KKT_NA_TPB) k_na_dual(long long n, long long m, const int64_t* __restrict__ rp,
                                                        const int32_t* __restrict__ ci, const double* __restrict__ v,
                                                        const double* __restrict__ c, const double* __restrict__ x,
                                                        const double* __restrict__ y, double* __restrict__ scratch) {
  double acc[5] = {0, 0, 0, 0, 0};
  const bool mx[5] = {false, true, false, false, false};
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long j = warp; j < n; j += nwarps) {
    const double g = na_row_dot(rp, ci, v, y, j, lane, m);
    if (lane == 0) {
      const double cj = c[j], xj = x[j];
      const double rd = na_relu(g - cj);
      acc[0] += rd * rd;
      acc[1] = fmax(acc[1], rd);
      acc[2] += cj * xj;
      acc[3] += xj * na_relu(cj - g);
      acc[4] += cj * cj;
    }
  }
  pdhg::block_reduce<5>(acc, mx);
  if (threadIdx.x == 0) {
    double* p = scratch + (size_t)blockIdx.x * KKT_NA_Q;
    p[NA_RD2] = acc[0];
    p[NA_RDINF] = acc[1];
    p[NA_CX] = acc[2];
    p[NA_XZ] = acc[3];
    p[NA_C2] = acc[4];
  }
}

__global__ void __launch_bounds__(KKT_NA_TPB) k_na_primal(long long m, long long n, const int64_t* __restrict__ rp,
                                                          const int32_t* __restrict__ ci,
                                                          const double* __restrict__ v, const double* __restrict__ b,
                                                          const double* __restrict__ x, const double* __restrict__ y,
                                                          double* __restrict__ scratch) {
  double acc[4] = {0, 0, 0, 0};
  const bool mx[4] = {false, true, false, false};
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long i = warp; i < m; i += nwarps) {
    const double h = na_row_dot(rp, ci, v, x, i, lane, n);
    if (lane == 0) {
      const double bi = b[i];
      const double r = bi - h;
      acc[0] += r * r;
      acc[1] = fmax(acc[1], fabs(r));
      acc[2] += bi * y[i];
      acc[3] += bi * bi;
    }
  }
  pdhg::block_reduce<4>(acc, mx);
  if (threadIdx.x == 0) {
    double* p = scratch + (size_t)blockIdx.x * KKT_NA_Q;
    p[NA_RP2] = acc[0];
    p[NA_RPINF] = acc[1];
    p[NA_BY] = acc[2];
    p[NA_B2] = acc[3];
  }
}

// warp q sums quantity q over the nb blocks in a fixed order
__global__ void k_na_finalize(int nb, double* __restrict__ scratch) {
  const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (q >= NA_COUNT) return;
  const bool is_max = (q == NA_RDINF || q == NA_RPINF);
  double acc = 0.0;
  for (int b = lane; b < nb; b += 32) {
    const double v = scratch[(size_t)b * KKT_NA_Q + q];
    acc = is_max ? fmax(acc, v) : acc + v;
  }
  acc = is_max ? pdhg::warp_max(acc) : pdhg::warp_sum(acc);
  if (lane == 0) scratch[KKT_NA_SCRATCH_DOUBLES + q] = acc;
#ifdef PDHG_CHECKED
  if (threadIdx.x == 0) {
    scratch[KKT_NA_SCRATCH_DOUBLES + NA_COUNT] = (double)g_na_check;
    g_na_check = 0u;
  }
#endif
}

// Device address of the scratch array on the current device, looked up once
// per device (the first call on each device does it).
cudaError_t scratch_address(int device, double** out) {
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_kkt_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[device] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[device];
  return cudaSuccess;
}

}  // namespace

// defined in pdhg_api.cu: the message pdhg_last_error(NULL) returns
void pdhg_set_global_error(const char* msg);

namespace {

pdhg_status na_fail(pdhg_status s, const char* msg) {
  pdhg_set_global_error(msg);
  return s;
}

}  // namespace

extern "C" {

PDHG_API pdhg_status pdhg_kkt_noalloc(int64_t m, int64_t n, const int64_t* a_row_ptr, const int32_t* a_col_idx,
                                      const double* a_val, const int64_t* at_row_ptr, const int32_t* at_col_idx,
                                      const double* at_val, const double* b, const double* c, const double* x,
                                      const double* y, int blocks, void* cuda_stream, pdhg_kkt_info* out) {
  if (!out) return na_fail(PDHG_ERR_INVALID, "out is NULL");
  if (m < 1 || n < 1 || m >= (1LL << 31) || n >= (1LL << 31))
    return na_fail(PDHG_ERR_INVALID, "m and n must be in [1, 2^31)");
  if (!a_row_ptr || !a_col_idx || !a_val || !at_row_ptr || !at_col_idx || !at_val || !b || !c || !x || !y)
    return na_fail(PDHG_ERR_INVALID, "NULL array argument");
  if (blocks < 0 || blocks > KKT_NA_MAX_BLOCKS)
    return na_fail(PDHG_ERR_INVALID, "blocks must be in [0, 1024]: the static scratch holds partial sums for at "
                                     "most 1024 blocks");
  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) return na_fail(PDHG_ERR_CUDA, cudaGetErrorString(e));
  if (device < 0 || device >= KKT_NA_MAX_DEVICES) return na_fail(PDHG_ERR_INVALID, "device index >= 64");
  double* scratch = nullptr;
  e = scratch_address(device, &scratch);
  if (e != cudaSuccess) return na_fail(PDHG_ERR_CUDA, cudaGetErrorString(e));
  int nb = blocks;
  if (nb == 0) {
    int sms = 148;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) return na_fail(PDHG_ERR_CUDA, cudaGetErrorString(e));
    nb = std::min(KKT_NA_MAX_BLOCKS, 4 * sms);
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  k_na_dual<<<nb, KKT_NA_TPB, 0, s>>>(n, m, at_row_ptr, at_col_idx, at_val, c, x, y, scratch);
  k_na_primal<<<nb, KKT_NA_TPB, 0, s>>>(m, n, a_row_ptr, a_col_idx, a_val, b, x, y, scratch);
  k_na_finalize<<<1, 32 * NA_COUNT, 0, s>>>(nb, scratch);
  double q[KKT_NA_Q];
  e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(q, scratch + KKT_NA_SCRATCH_DOUBLES, sizeof(double) * (NA_COUNT + 1), cudaMemcpyDeviceToHost,
                        s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return na_fail(PDHG_ERR_CUDA, cudaGetErrorString(e));
#ifdef PDHG_CHECKED
  if (q[NA_COUNT] != 0.0)
    return na_fail(PDHG_ERR_INVALID, "checked build: a column index outside its vector was found and skipped");
#endif
  out->rp_norm2 = sqrt(q[NA_RP2]);
  out->rp_norminf = q[NA_RPINF];
  out->rd_norm2 = sqrt(q[NA_RD2]);
  out->rd_norminf = q[NA_RDINF];
  out->primal_obj = q[NA_CX];
  out->dual_obj = q[NA_BY];
  out->gap = fabs(q[NA_CX] - q[NA_BY]);
  out->complementarity = q[NA_XZ];
  out->rel_p = out->rp_norm2 / (1.0 + sqrt(q[NA_B2]));
  out->rel_d = out->rd_norm2 / (1.0 + sqrt(q[NA_C2]));
  out->rel_gap = out->gap / (1.0 + fabs(out->primal_obj) + fabs(out->dual_obj));
  out->rel_kkt = std::max(out->rel_p, std::max(out->rel_d, out->rel_gap));
  out->iteration = -1;
  // std::max and the fmax of the reductions drop a NaN operand, so rel_kkt
  // alone can look finite while a term is not: every sum is checked
  bool finite = true;
  for (int i = 0; i < NA_COUNT; ++i) finite = finite && std::isfinite(q[i]);
  if (!finite || !std::isfinite(out->rel_p) || !std::isfinite(out->rel_d) || !std::isfinite(out->rel_gap))
    return na_fail(PDHG_ERR_NUMERIC, "NaN or Inf in the KKT measures");
  return PDHG_OK;
}

}  // extern "C"
