// hz_launch.cu -- launch shapes (occupancy-derived grids), variant tables and
// the stand-alone deterministic dot product.
#include <map>
#include <mutex>
#include <utility>

#include "hz_krylov.cuh"

namespace hz {

namespace {
std::mutex g_occ_mu;
std::map<std::pair<const void*, size_t>, int> g_occ;  // blocks per SM of each (kernel, dynamic smem)
}  // namespace

int grid_for(const void* kernel, int block, const Launch& L, int64_t work_blocks, size_t smem, int per_sm_cap) {
  int per_sm = 0;
  {
    std::lock_guard<std::mutex> lk(g_occ_mu);
    const auto key = std::make_pair(kernel, smem);
    auto it = g_occ.find(key);
    if (it != g_occ.end()) {
      per_sm = it->second;
    } else {
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
      }
      g_occ[key] = per_sm;
    }
  }
  if (per_sm_cap > 0 && per_sm > per_sm_cap) per_sm = per_sm_cap;
  int64_t gsz = (int64_t)per_sm * L.sms;
  if (gsz > work_blocks) gsz = work_blocks;
  if (gsz > kMaxGrid) gsz = kMaxGrid;
  return gsz < 1 ? 1 : (int)gsz;
}

void warm_launch_kernels(const Launch& L);  // hz_setup.cu

template <typename T>
__global__ void __launch_bounds__(256) k_dot(int64_t n, const T* __restrict__ x, const T* __restrict__ y, Red red,
                                             double* out_dev) {
  double acc = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    acc += (double)x[e] * (double)y[e];
  double vv[1] = {acc}, out[1];
  if (grid_reduce<1>(vv, red, out)) *out_dev = out[0];
}

template <typename T>
cudaError_t launch_dot(int64_t n, const T* x, const T* y, Red red, double* out_dev, int grid, cudaStream_t s) {
  k_dot<T><<<grid, 256, 0, s>>>(n, x, y, red, out_dev);
  return cudaGetLastError();
}
template cudaError_t launch_dot<float>(int64_t, const float*, const float*, Red, double*, int, cudaStream_t);
template cudaError_t launch_dot<double>(int64_t, const double*, const double*, Red, double*, int, cudaStream_t);

void warm_launch_cache(const Launch& L) {
  warm_kernels<float>(L);
  warm_kernels<double>(L);
  warm_sor<float>(L);
  warm_sor<double>(L);
  warm_launch_kernels(L);
}

int num_variants(int prec, int kind) {
  if (prec == 0) return kind == 0 ? Variants<float>::NPRE : Variants<float>::NMV;
  return kind == 0 ? Variants<double>::NPRE : Variants<double>::NMV;
}

bool variant_parks_smem(int prec, int kind, int id) {
  if (kind != 0) return false;
  return (prec == 0 ? Variants<float>::pre_p[id] : Variants<double>::pre_p[id]) == PARK_SMEM;
}

void variant_flags(int prec, int kind, int id, int* l2, int* cap) {
  if (kind == 0) {
    *l2 = (prec == 0 ? Variants<float>::pre_p[id] : Variants<double>::pre_p[id]) == PARK_OUT_L2;
    *cap = prec == 0 ? Variants<float>::pre_b[id] : Variants<double>::pre_b[id];
  } else {
    *l2 = prec == 0 ? Variants<float>::mv_h[id] : Variants<double>::mv_h[id];
    *cap = prec == 0 ? Variants<float>::mv_b[id] : Variants<double>::mv_b[id];
  }
}

int variant_park_mode(int prec, int id) {
  return prec == 0 ? Variants<float>::pre_p[id] : Variants<double>::pre_p[id];
}

void variant_shape(int prec, int kind, int id, int* vec, int* depth) {
  if (prec == 0) {
    *vec = kind == 0 ? Variants<float>::pre_v[id] : Variants<float>::mv_v[id];
    *depth = kind == 0 ? Variants<float>::pre_u[id] : Variants<float>::mv_u[id];
  } else {
    *vec = kind == 0 ? Variants<double>::pre_v[id] : Variants<double>::mv_v[id];
    *depth = kind == 0 ? Variants<double>::pre_u[id] : Variants<double>::mv_u[id];
  }
}

}  // namespace hz

// ---------------------------------------------------------------------------
// hz_dot_noalloc: the deterministic dot product with its scratch in static
// device memory instead of memory the library allocates.
//
// For callers that cannot allocate device memory (code that runs where
// cudaMalloc is not allowed or not wanted: inside a memory pool that must not
// grow, in a process whose allocator is owned by someone else, or under a
// strict no-allocation policy after start-up).  The scratch is one
// file-scope array: HZ_DOT_NOALLOC_SLOTS FP64 partial sums (one per block)
// plus a ticket word, 32 KiB in all, which every GPU that loads the library
// holds until the process exits.
namespace {
constexpr int kNoAllocSlots = HZ_DOT_NOALLOC_SLOTS;
static __device__ __align__(256) double hz_noalloc_scratch[kNoAllocSlots + 32];

std::mutex g_na_mu;
double* g_na_ptr[64] = {};  // device address of the scratch, per device (set up once)
}  // namespace

extern "C" int hz_dot_noalloc(int prec, int64_t n, const void* x, const void* y, void* stream, double* out) {
  using namespace hz;
  if (n < 0 || !out || (n > 0 && (!x || !y))) return HZ_ERR_INVALID;
  if (prec != HZ_PREC_FP32 && prec != HZ_PREC_FP64) return HZ_ERR_INVALID;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return HZ_ERR_CUDA;
  double* base = nullptr;
  {
    // set-up, once per device with that device current: the host-side name of
    // the array is not a device address, so ask the runtime for the address
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, hz_noalloc_scratch) != cudaSuccess) return HZ_ERR_CUDA;
      g_na_ptr[dev] = (double*)p;
    }
    base = g_na_ptr[dev];
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return HZ_ERR_CUDA;
  int64_t grid = (int64_t)sms * 8;
  if (grid > kNoAllocSlots) grid = kNoAllocSlots;  // grid-stride: fewer blocks than SMs*8 is still correct
  const int64_t need = (n + 255) / 256;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned* ticket = reinterpret_cast<unsigned*>(base + kNoAllocSlots);
  // the ticket must start at zero whatever the previous call left
  if (cudaMemsetAsync(ticket, 0, sizeof(unsigned), s) != cudaSuccess) return HZ_ERR_CUDA;
  if (n == 0) return cudaMemsetAsync(out, 0, sizeof(double), s) == cudaSuccess ? HZ_OK : HZ_ERR_CUDA;
  Red red{base, ticket};
  cudaError_t e = prec == HZ_PREC_FP32
                      ? launch_dot<float>(n, (const float*)x, (const float*)y, red, out, (int)grid, s)
                      : launch_dot<double>(n, (const double*)x, (const double*)y, red, out, (int)grid, s);
  return e == cudaSuccess ? HZ_OK : HZ_ERR_CUDA;
}
