// hz_launch.cu -- launch shapes (occupancy-derived grids), variant tables and
// the stand-alone deterministic dot product.
#include <mutex>
#include <unordered_map>

#include "hz_krylov.cuh"

namespace hz {

namespace {
std::mutex g_occ_mu;
std::unordered_map<const void*, int> g_occ;  // blocks per SM of each kernel at its block size
}  // namespace

int grid_for(const void* kernel, int block, const Launch& L, int64_t work_blocks) {
  int per_sm = 0;
  {
    std::lock_guard<std::mutex> lk(g_occ_mu);
    auto it = g_occ.find(kernel);
    if (it != g_occ.end()) {
      per_sm = it->second;
    } else {
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, 0) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
      }
      g_occ[kernel] = per_sm;
    }
  }
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
  warm_launch_kernels(L);
}

int num_variants(int prec, int kind) {
  if (prec == 0) return kind == 0 ? Variants<float>::NPRE : Variants<float>::NMV;
  return kind == 0 ? Variants<double>::NPRE : Variants<double>::NMV;
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
