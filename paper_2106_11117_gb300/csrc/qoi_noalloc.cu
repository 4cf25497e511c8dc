// QoI reduction that allocates no memory (lflts_qoi_reduce_noalloc).
//
// The regular path (lflts_solve) keeps its QoI partial sums in workspace
// buffers that the context allocates with cudaMalloc.  Some callers cannot
// let a library allocate: applications whose device memory is owned by their
// own pool allocator (a library cudaMalloc would fragment or exceed its
// budget), or code that must not allocate once it is running (fixed memory
// plans, latency-bound loops where a cudaMalloc would synchronise the device).
// This entry point runs the same two-stage compensated reduction with its
// partial sums in a fixed-size array that lives in the library's device
// image, so the call itself performs no allocation.
//
// The array below is part of the module: every GPU that loads the library
// holds it (2 MiB) until the process exits.  All calls on a device share it.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/lflts.h"

namespace {

constexpr int kChunk = 512;                                 // weights per stage-1 block (as lflts_solve)
constexpr int64_t kScratchDoubles = int64_t(1) << 18;      // 2 MiB of FP64
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

// Device address of g_noalloc_scratch per device.  In host code the symbol
// is only a host-side stand-in, so the address must come from
// cudaGetSymbolAddress, called with that device current.
void* g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

// Compensated (Neumaier) FP64 accumulator; the same summation order as the
// QoI reduction of lflts_solve: weights in chunks of 512 in index order,
// then the chunk partials in chunk order.
struct Acc {
  double s = 0.0, c = 0.0;
  __device__ __forceinline__ void add(double x) {
    const double t = s + x;
    if (fabs(s) >= fabs(x)) c += (s - t) + x;
    else c += (x - t) + s;
    s = t;
  }
};

template <typename Real>
__global__ void k_qoi_partial_noalloc(const Real* __restrict__ u, int64_t n_rows, int S,
                                      const int* __restrict__ idx, const double* __restrict__ gw, int nnz,
                                      double* __restrict__ ps, double* __restrict__ pc) {
  const int s = blockIdx.y * blockDim.x + threadIdx.x;
  if (s >= S) return;
  const int c = blockIdx.x;
  const int k0 = c * kChunk, k1 = min(nnz, k0 + kChunk);
  Acc acc;
  for (int k = k0; k < k1; ++k) {
    const int r = idx[k];
    if (r < 0 || r >= n_rows) continue;  // out-of-range rows are skipped, never read
    acc.add(__dmul_rn(gw[k], (double)u[(size_t)r * S + s]));  // rounded alone, as in lflts_solve
  }
  ps[(size_t)c * S + s] = acc.s;
  pc[(size_t)c * S + s] = acc.c;
}

__global__ void k_qoi_final_noalloc(int n_chunks, int S, const double* __restrict__ ps,
                                    const double* __restrict__ pc, double* __restrict__ Q) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  Acc acc;
  for (int c = 0; c < n_chunks; ++c) {
    acc.add(ps[(size_t)c * S + s]);
    acc.c += pc[(size_t)c * S + s];
  }
  Q[s] = acc.s + acc.c;
}

}  // namespace

// Defined in lflts.cu: stores a message in the context (ctx may be NULL);
// the device of a context (-1 for a host-only context).
int lflts_internal_set_error(lflts_ctx* ctx, int code, const char* msg);
int lflts_internal_ctx_device(const lflts_ctx* ctx);

extern "C" int lflts_qoi_reduce_noalloc(lflts_ctx* ctx, const void* u, int precision, int64_t n_rows,
                                        int64_t S, const int32_t* idx, const double* g, int64_t nnz,
                                        double* Q, void* stream) {
  if (!u || !idx || !g || !Q || S < 1 || n_rows < 1 || nnz < 1 || nnz >= INT32_MAX || S >= INT32_MAX ||
      (precision != 32 && precision != 64))
    return lflts_internal_set_error(ctx, LFLTS_ERR_ARG,
                                    "qoi_reduce_noalloc: null pointer, empty size or precision not 32/64");
  const int64_t n_chunks = (nnz + kChunk - 1) / kChunk;
  if (2 * n_chunks * S > kScratchDoubles)
    return lflts_internal_set_error(
        ctx, LFLTS_ERR_ARG,
        ("qoi_reduce_noalloc: ceil(nnz/512) * S = " + std::to_string(n_chunks * S) +
         " exceeds the fixed scratch capacity of " + std::to_string(kScratchDoubles / 2) + " partial sums")
            .c_str());
  // the context's device when there is one, else the current device
  const int cdev = ctx ? lflts_internal_ctx_device(ctx) : -1;
  if (cdev >= 0 && cudaSetDevice(cdev) != cudaSuccess)
    return lflts_internal_set_error(ctx, LFLTS_ERR_CUDA, "qoi_reduce_noalloc: cannot select the context's device");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return lflts_internal_set_error(ctx, LFLTS_ERR_CUDA, "qoi_reduce_noalloc: no current device");
  void* scratch = nullptr;
  {
    // once per device, with that device current: resolve the array's address
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p)
        return lflts_internal_set_error(
            ctx, LFLTS_ERR_CUDA,
            (std::string("qoi_reduce_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e)).c_str());
      g_scratch_ptr[dev] = p;
    }
    scratch = g_scratch_ptr[dev];
  }
  double* ps = static_cast<double*>(scratch);
  double* pc = ps + n_chunks * S;  // every slot of both halves is written before it is read
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int tb = static_cast<int>(S < 128 ? S : 128);
  const dim3 grid1(static_cast<unsigned>(n_chunks), static_cast<unsigned>((S + tb - 1) / tb));
  if (precision == 32)
    k_qoi_partial_noalloc<float><<<grid1, tb, 0, st>>>(static_cast<const float*>(u), n_rows, (int)S, idx, g,
                                                        (int)nnz, ps, pc);
  else
    k_qoi_partial_noalloc<double><<<grid1, tb, 0, st>>>(static_cast<const double*>(u), n_rows, (int)S, idx, g,
                                                         (int)nnz, ps, pc);
  e = cudaGetLastError();
  if (e != cudaSuccess)
    return lflts_internal_set_error(ctx, LFLTS_ERR_CUDA,
                                    (std::string("qoi_reduce_noalloc: ") + cudaGetErrorString(e)).c_str());
  k_qoi_final_noalloc<<<static_cast<unsigned>((S + 127) / 128), 128, 0, st>>>((int)n_chunks, (int)S, ps, pc, Q);
  e = cudaGetLastError();
  if (e != cudaSuccess)
    return lflts_internal_set_error(ctx, LFLTS_ERR_CUDA,
                                    (std::string("qoi_reduce_noalloc: ") + cudaGetErrorString(e)).c_str());
  return LFLTS_OK;
}
