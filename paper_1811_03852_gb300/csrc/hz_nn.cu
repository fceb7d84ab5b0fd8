// hz_nn.cu -- the learned preconditioner stage: a 4-layer 3-D conv net
// (1 -> 16 -> 16 -> 16 -> 1 channels, 3x3x3 kernels, exact-erf GELU after the
// first three layers), its inference inside the flexible Krylov solver, and
// its training (backward pass, deterministic weight-gradient reduction, Adam).
//
// Convolution = cross-correlation with bias:
//   y[o, p] = b[o] + sum_{c, tap} W[o][c][tap] x[c, p + tap],  tap = (dk, dj, di) in {-1,0,1}^3,
// with zero padding in k (levels) and j (latitude; also at the edges of
// stacked training crops, every seg_ny rows) and periodic wrap in i
// (longitude) for full fields or zero padding for crops.
//
// Precision: weights and stored activations BF16, every sum accumulated in
// FP32.  The 16 -> 16 layers run on the tensor cores (mma.sync m16n8k16 BF16,
// FP32 accumulate; a warp computes 16 points x 16 output channels per tile,
// one MMA k-step per tap).  The 1 -> 16 and 16 -> 1 layers and the whole
// backward pass (FP32 activation gradients) run on the CUDA cores.
// Activations are channel-last: [point][16], point = (k*ny + j)*nx + i.
#include <cuda_bf16.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "hz_nn.cuh"

namespace hz {

// flat parameter layout (per layer W[Cout][Cin][27] then b[Cout])
constexpr int kP1 = kC * 1 * kTaps, kP2 = kC * kC * kTaps, kP4 = 1 * kC * kTaps;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kP1;
constexpr int kOffW2 = kOffB1 + kC, kOffB2 = kOffW2 + kP2;
constexpr int kOffW3 = kOffB2 + kC, kOffB3 = kOffW3 + kP2;
constexpr int kOffW4 = kOffB3 + kC, kOffB4 = kOffW4 + kP4;
constexpr int kNParams = kOffB4 + 1;

// index of the neighbour of (i, j, k) at tap t, or -1 outside the domain
__device__ __forceinline__ int64_t nbr(const NnGrid& g, int i, int j, int k, int t) {
  const int dk = t / 9 - 1, dj = (t / 3) % 3 - 1, di = t % 3 - 1;
  const int kk = k + dk;
  if (kk < 0 || kk >= g.nz) return -1;
  if (dj == -1 && (j % g.seg) == 0) return -1;
  if (dj == 1 && (j % g.seg) == g.seg - 1) return -1;
  const int jj = j + dj;
  int ii = i + di;
  if (ii < 0 || ii >= g.nx) {
    if (!g.periodic) return -1;
    ii = ii < 0 ? ii + g.nx : ii - g.nx;
  }
  return ((int64_t)kk * g.ny + jj) * g.nx + ii;
}

// ---- layer 1: x (FP32, one channel, scaled by s) -> z1 (FP32, optional), h1 = gelu(z1) (BF16)
__global__ void __launch_bounds__(256) k_nn_l1(NnGrid g, const float* __restrict__ x, const double* scale_nrm2,
                                               float scale, NnW w, float* __restrict__ z, __nv_bfloat16* __restrict__ h) {
  __shared__ float W[kTaps * kC + kC];
  for (int q = threadIdx.x; q < kTaps * kC; q += blockDim.x) W[q] = w.w1[q];
  for (int q = threadIdx.x; q < kC; q += blockDim.x) W[kTaps * kC + q] = w.b1[q];
  __syncthreads();
  float s = scale;
  if (scale_nrm2) {  // input scaled by 1/sigma, sigma = rms of the field
    const double v = *scale_nrm2;
    s = v > 0.0 ? (float)(1.0 / sqrt(v / (double)g.n)) : 0.f;
  }
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < g.n; p += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(p % g.nx), j = (int)((p / g.nx) % g.ny), k = (int)(p / ((int64_t)g.nx * g.ny));
    float acc[kC];
#pragma unroll
    for (int c = 0; c < kC; ++c) acc[c] = W[kTaps * kC + c];
    for (int t = 0; t < kTaps; ++t) {
      const int64_t q = nbr(g, i, j, k, t);
      const float xv = q >= 0 ? s * x[q] : 0.f;
#pragma unroll
      for (int c = 0; c < kC; ++c) acc[c] = fmaf(W[t * kC + c], xv, acc[c]);
    }
    if (z) {
#pragma unroll
      for (int c = 0; c < kC; c += 4) *reinterpret_cast<float4*>(z + p * kC + c) = make_float4(acc[c], acc[c + 1], acc[c + 2], acc[c + 3]);
    }
    __align__(16) __nv_bfloat16 hv[kC];
#pragma unroll
    for (int c = 0; c < kC; ++c) hv[c] = __float2bfloat16_rn(gelu_f(acc[c]));
    reinterpret_cast<uint4*>(h + p * kC)[0] = reinterpret_cast<const uint4*>(hv)[0];
    reinterpret_cast<uint4*>(h + p * kC)[1] = reinterpret_cast<const uint4*>(hv)[1];
  }
}

// ---- layers 2, 3: 16 -> 16 on the tensor cores ------------------------------
__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// A warp computes a tile of 16 consecutive points of one row (k, j) for all 16
// output channels: for every tap, A = the 16 x 16 (point x input channel)
// neighbours, B = W[tap] (input channel x output channel); two n8 halves.
// Fragment layout of m16n8k16 (g = lane/4, c = lane%4): A rows g, g+8 and
// columns 2c, 2c+1, 2c+8, 2c+9; B rows (k) 2c, 2c+1, 2c+8, 2c+9 of column g;
// D rows g, g+8, columns 2c, 2c+1.
__global__ void __launch_bounds__(128) k_nn_mid(NnGrid g, const __nv_bfloat16* __restrict__ hin,
                                               const __nv_bfloat16* __restrict__ wb, const float* __restrict__ bias,
                                               float* __restrict__ z, __nv_bfloat16* __restrict__ hout) {
  __shared__ uint32_t Ws[kTaps * kC * kC / 2];  // [tap][co][ci] bf16 pairs
  __shared__ float Bs[kC];
  for (int q = threadIdx.x; q < kTaps * kC * kC / 2; q += blockDim.x) Ws[q] = reinterpret_cast<const uint32_t*>(wb)[q];
  for (int q = threadIdx.x; q < kC; q += blockDim.x) Bs[q] = bias[q];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, gq = lane >> 2, cq = lane & 3;
  const int tiles_row = (g.nx + 15) / 16;
  const int64_t ntiles = (int64_t)tiles_row * g.ny * g.nz;
  const int64_t wstride = (int64_t)gridDim.x * (blockDim.x >> 5);
  const uint32_t* hin32 = reinterpret_cast<const uint32_t*>(hin);
  for (int64_t tile = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; tile < ntiles; tile += wstride) {
    const int it = (int)(tile % tiles_row);
    const int64_t row = tile / tiles_row;  // k*ny + j
    const int j = (int)(row % g.ny), k = (int)(row / g.ny);
    const int i0 = it * 16;
    const int ia = i0 + gq, ib = i0 + gq + 8;  // the two points this lane feeds
    float d0[4], d1[4];
    d0[0] = d0[2] = Bs[2 * cq];
    d0[1] = d0[3] = Bs[2 * cq + 1];
    d1[0] = d1[2] = Bs[8 + 2 * cq];
    d1[1] = d1[3] = Bs[8 + 2 * cq + 1];
    for (int t = 0; t < kTaps; ++t) {
      const int64_t qa = ia < g.nx ? nbr(g, ia, j, k, t) : -1;
      const int64_t qb = ib < g.nx ? nbr(g, ib, j, k, t) : -1;
      uint32_t a[4];
      a[0] = qa >= 0 ? hin32[qa * (kC / 2) + cq] : 0u;
      a[1] = qb >= 0 ? hin32[qb * (kC / 2) + cq] : 0u;
      a[2] = qa >= 0 ? hin32[qa * (kC / 2) + 4 + cq] : 0u;
      a[3] = qb >= 0 ? hin32[qb * (kC / 2) + 4 + cq] : 0u;
      const uint32_t* wt = Ws + t * (kC * kC / 2);
      // B[k = ci][n = co] = W[t][co][ci]: ci pairs (2c, 2c+1) and (2c+8, 2c+9) of column co = g (+8)
      mma_bf16_16816(d0, a, wt[gq * (kC / 2) + cq], wt[gq * (kC / 2) + 4 + cq]);
      mma_bf16_16816(d1, a, wt[(gq + 8) * (kC / 2) + cq], wt[(gq + 8) * (kC / 2) + 4 + cq]);
    }
    // epilogue: point ia gets d*[0..1], point ib gets d*[2..3]; channels 2c, 2c+1 and 8+2c, 9+2c
    const int64_t pbase = row * g.nx;
    if (ia < g.nx) {
      const int64_t p = pbase + ia;
      if (z) {
        *reinterpret_cast<float2*>(z + p * kC + 2 * cq) = make_float2(d0[0], d0[1]);
        *reinterpret_cast<float2*>(z + p * kC + 8 + 2 * cq) = make_float2(d1[0], d1[1]);
      }
      reinterpret_cast<__nv_bfloat162*>(hout + p * kC + 2 * cq)[0] = __floats2bfloat162_rn(gelu_f(d0[0]), gelu_f(d0[1]));
      reinterpret_cast<__nv_bfloat162*>(hout + p * kC + 8 + 2 * cq)[0] = __floats2bfloat162_rn(gelu_f(d1[0]), gelu_f(d1[1]));
    }
    if (ib < g.nx) {
      const int64_t p = pbase + ib;
      if (z) {
        *reinterpret_cast<float2*>(z + p * kC + 2 * cq) = make_float2(d0[2], d0[3]);
        *reinterpret_cast<float2*>(z + p * kC + 8 + 2 * cq) = make_float2(d1[2], d1[3]);
      }
      reinterpret_cast<__nv_bfloat162*>(hout + p * kC + 2 * cq)[0] = __floats2bfloat162_rn(gelu_f(d0[2]), gelu_f(d0[3]));
      reinterpret_cast<__nv_bfloat162*>(hout + p * kC + 8 + 2 * cq)[0] = __floats2bfloat162_rn(gelu_f(d1[2]), gelu_f(d1[3]));
    }
  }
}

// ---- layer 4: h3 (BF16, 16 channels) -> y (FP32).  With base != null the
// preconditioner combination out = base + sigma * y is written instead, sigma
// = rms of the stage input (sqrt(nrm2 / n)).
__global__ void __launch_bounds__(256) k_nn_l4(NnGrid g, const __nv_bfloat16* __restrict__ h, NnW w,
                                               const float* base, const double* nrm2, float* out) {
  __shared__ float W[kTaps * kC + 1];
  for (int q = threadIdx.x; q < kTaps * kC; q += blockDim.x) W[q] = w.w4[q];
  if (threadIdx.x == 0) W[kTaps * kC] = w.b4[0];
  __syncthreads();
  float sigma = 1.f;
  if (nrm2) {
    const double v = *nrm2;
    sigma = (float)sqrt(v / (double)g.n);
  }
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < g.n; p += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(p % g.nx), j = (int)((p / g.nx) % g.ny), k = (int)(p / ((int64_t)g.nx * g.ny));
    float acc = W[kTaps * kC];
    for (int t = 0; t < kTaps; ++t) {
      const int64_t q = nbr(g, i, j, k, t);
      if (q < 0) continue;
      __align__(16) __nv_bfloat16 hv[kC];
      reinterpret_cast<uint4*>(hv)[0] = reinterpret_cast<const uint4*>(h + q * kC)[0];
      reinterpret_cast<uint4*>(hv)[1] = reinterpret_cast<const uint4*>(h + q * kC)[1];
#pragma unroll
      for (int c = 0; c < kC; ++c) acc = fmaf(W[t * kC + c], __bfloat162float(hv[c]), acc);
    }
    out[p] = base ? fmaf(sigma, acc, base[p]) : acc;
  }
}

// ---- plane-tiled forward kernels ----------------------------------------------
// A block owns a kTI x kTJ tile of columns (i, j) and marches k.  A ring of
// four shared-memory planes holds the input at levels k-1, k, k+1 (with a
// one-point halo in i and j) while cp.async fetches level k+2, so every tap
// of the 3x3x3 stencil is read from shared memory and each input value
// leaves HBM once per tile.  Halo points outside the domain, across a crop
// seam (every seg rows) or past the periodic wrap are zero-filled by the copy.
// Used when no tile straddles a crop seam (seg a multiple of kTJ, or one
// segment); the gather kernels above handle the rest.
constexpr int kTI = 32, kTJ = 4;
constexpr int kPI = kTI + 2, kPJ = kTJ + 2, kPP = kPI * kPJ;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem, int src_bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

struct TileGeo {
  int i0, j0;
  bool jlo_zero, jhi_zero;  // the halo row above / below lies across a crop seam
};

__device__ __forceinline__ TileGeo tile_geo(const NnGrid& g, int64_t tile, int tiles_i) {
  TileGeo t;
  t.i0 = (int)(tile % tiles_i) * kTI;
  t.j0 = (int)(tile / tiles_i) * kTJ;
  t.jlo_zero = (t.j0 % g.seg) == 0;
  t.jhi_zero = ((t.j0 + kTJ) % g.seg) == 0;
  return t;
}

// source point of plane position (ti, tj) at level k, or -1 for a zero
__device__ __forceinline__ int64_t plane_src(const NnGrid& g, const TileGeo& t, int k, int ti, int tj) {
  if (k < 0 || k >= g.nz) return -1;
  if ((tj == 0 && t.jlo_zero) || (tj == kPJ - 1 && t.jhi_zero)) return -1;
  const int gj = t.j0 - 1 + tj;
  if (gj < 0 || gj >= g.ny) return -1;
  int gi = t.i0 - 1 + ti;
  if (gi < 0) {
    if (!g.periodic) return -1;
    gi += g.nx;
  } else if (gi >= g.nx) {
    if (!g.periodic) return -1;
    gi -= g.nx;
  }
  if (gi < 0 || gi >= g.nx) return -1;
  return ((int64_t)k * g.ny + gj) * g.nx + gi;
}

// 16-channel BF16 planes hold one 16-byte chunk per point and half
// (channels 0-7 in [0], 8-15 in [1]): the eight rows of an ldmatrix (eight
// consecutive points of one half) are 128 contiguous bytes, so they hit
// distinct banks.
__device__ __forceinline__ void ldmatrix_x4(uint32_t (&r)[4], unsigned saddr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(saddr));
}

// Shared-memory address of this lane's ldmatrix row for the A fragment (16
// points x 16 channels) of output row w, points 16*mt .. 16*mt+15 of the tile,
// unshifted: tap (dj, di) adds (dj * kPI + di) * 16 bytes.
__device__ __forceinline__ unsigned a_row_addr(uint4 (*pl)[kPP], int w, int mt, int lane) {
  const int mi = lane >> 3, r = lane & 7;
  const int pp = (w + 1) * kPI + 16 * mt + (mi & 1) * 8 + r + 1;
  return (unsigned)__cvta_generic_to_shared(&pl[mi >> 1][pp]);
}
constexpr unsigned kSlotBytes = 2 * kPP * 16;  // one ring slot: both halves of a plane
__device__ __forceinline__ constexpr int tap_off(int tp) {
  return (((tp / 3) % 3 - 1) * kPI + (tp % 3 - 1)) * 16;
}

// Per-thread copy list of one tile's plane: the chunks this thread copies
// (point pp, half h), as the source element offset within one level (-1: zero
// fill) and the destination byte offset within a ring slot.  Built once per
// tile; a level adds k * ny * nx.
template <int NCH, int BYTES>
struct PlaneCopy {
  static constexpr int kMax = (NCH * kPP + kTI * kTJ - 1) / (kTI * kTJ);
  int64_t src[kMax];
  unsigned dst[kMax];
  __device__ __forceinline__ void init(const NnGrid& g, const TileGeo& t) {
#pragma unroll
    for (int m = 0; m < kMax; ++m) {
      const int q = threadIdx.x + m * kTI * kTJ;
      src[m] = -2;
      if (q < NCH * kPP) {
        const int pp = q / NCH, hh = q % NCH;
        const int64_t s = plane_src(g, t, 0, pp % kPI, pp / kPI);
        src[m] = s >= 0 ? s * (NCH * BYTES / (NCH == 2 ? 2 : 4)) + hh * 8 : -1;
        dst[m] = (unsigned)((hh * kPP + pp) * BYTES);
      }
    }
  }
  // elements: bf16 units for NCH = 2 (16 channels, 16-byte chunks), float units for NCH = 1
  template <typename E>
  __device__ __forceinline__ void issue(unsigned slot, const E* base, int64_t kofs) const {
#pragma unroll
    for (int m = 0; m < kMax; ++m) {
      if (src[m] == -2) continue;
      const bool ok = src[m] >= 0;
      const void* gp = ok ? (const void*)(base + kofs + src[m]) : (const void*)base;
      if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(slot + dst[m]), "l"(gp), "r"(ok ? 16 : 0)
                     : "memory");
      else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(slot + dst[m]), "l"(gp), "r"(ok ? 4 : 0)
                     : "memory");
    }
  }
};

__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// The ring: kRing slots; output level k reads levels k-1, k, k+1 while the
// copies of k+2 (issued one level earlier) land and those of k+3 start.
constexpr int kRing = 5;

// layer 1 on planes: x (FP32, one channel) -> z1 (optional), h1 = gelu(z1).
// Same arithmetic order as k_nn_l1 (taps 0..26, one FMA each).
__global__ void __launch_bounds__(kTI * kTJ) k_nn_l1t(NnGrid g, const float* __restrict__ x, const double* scale_nrm2,
                                                    NnW w, float* __restrict__ z, __nv_bfloat16* __restrict__ h) {
  __shared__ __align__(16) float W[kTaps * kC + kC];
  __shared__ __align__(16) float pl[kRing][kPP];
  for (int q = threadIdx.x; q < kTaps * kC; q += blockDim.x) W[q] = w.w1[q];
  for (int q = threadIdx.x; q < kC; q += blockDim.x) W[kTaps * kC + q] = w.b1[q];
  float s = 1.f;
  if (scale_nrm2) {
    const double v = *scale_nrm2;
    s = v > 0.0 ? (float)(1.0 / sqrt(v / (double)g.n)) : 0.f;
  }
  const int tiles_i = (g.nx + kTI - 1) / kTI;
  const int64_t ntiles = (int64_t)tiles_i * ((g.ny + kTJ - 1) / kTJ);
  const int ti = threadIdx.x % kTI, tj = threadIdx.x / kTI;
  const int64_t plane = (int64_t)g.nx * g.ny;
  const unsigned sbase = (unsigned)__cvta_generic_to_shared(&pl[0][0]);
  constexpr unsigned kSlot = kPP * 4;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const TileGeo t = tile_geo(g, tile, tiles_i);
    PlaneCopy<1, 4> pc;
    pc.init(g, t);
    __syncthreads();  // previous tile's readers are done
    for (int kq = 0; kq < 3; ++kq) {
      if (kq < g.nz) pc.issue(sbase + kq * kSlot, x, kq * plane);
      cp_async_commit();
    }
    cp_async_wait_one();  // levels 0 and 1 landed
    __syncthreads();
    const int gi = t.i0 + ti, gj = t.j0 + tj;
    const bool valid = gi < g.nx && gj < g.ny;
    const int me = (tj + 1) * kPI + ti + 1;
    for (int k = 0; k < g.nz; ++k) {
      if (k + 3 < g.nz) pc.issue(sbase + ((k + 3) % kRing) * kSlot, x, (int64_t)(k + 3) * plane);
      cp_async_commit();
      const float* sp[3] = {pl[(k + kRing - 1) % kRing], pl[k % kRing], pl[(k + 1) % kRing]};
      const bool has[3] = {k > 0, true, k + 1 < g.nz};
      float acc[kC];
#pragma unroll
      for (int c = 0; c < kC; ++c) acc[c] = W[kTaps * kC + c];
#pragma unroll
      for (int tp = 0; tp < kTaps; ++tp) {
        const int dk = tp / 9, dj = (tp / 3) % 3 - 1, di = tp % 3 - 1;
        const float xv = has[dk] ? s * sp[dk][me + dj * kPI + di] : 0.f;
#pragma unroll
        for (int c4 = 0; c4 < kC / 4; ++c4) {
          const float4 wv = reinterpret_cast<const float4*>(W)[tp * (kC / 4) + c4];
          acc[4 * c4 + 0] = fmaf(wv.x, xv, acc[4 * c4 + 0]);
          acc[4 * c4 + 1] = fmaf(wv.y, xv, acc[4 * c4 + 1]);
          acc[4 * c4 + 2] = fmaf(wv.z, xv, acc[4 * c4 + 2]);
          acc[4 * c4 + 3] = fmaf(wv.w, xv, acc[4 * c4 + 3]);
        }
      }
      if (valid) {
        const int64_t p = (int64_t)k * plane + (int64_t)gj * g.nx + gi;
        if (z) {
#pragma unroll
          for (int c = 0; c < kC; c += 4)
            *reinterpret_cast<float4*>(z + p * kC + c) = make_float4(acc[c], acc[c + 1], acc[c + 2], acc[c + 3]);
        }
        __align__(16) __nv_bfloat16 hv[kC];
#pragma unroll
        for (int c = 0; c < kC; ++c) hv[c] = __float2bfloat16_rn(gelu_f(acc[c]));
        reinterpret_cast<uint4*>(h + p * kC)[0] = reinterpret_cast<const uint4*>(hv)[0];
        reinterpret_cast<uint4*>(h + p * kC)[1] = reinterpret_cast<const uint4*>(hv)[1];
      }
      cp_async_wait_one();  // level k+2 landed (k+3 may still be in flight)
      __syncthreads();
    }
  }
  cp_async_wait_all();
}

// layers 2, 3 on planes: 16 -> 16 on the tensor cores.  Warp w computes output
// row w of the tile (two 16-point m-tiles, both 8-channel n-halves); per tap
// one ldmatrix per m-tile and one m16n8k16 MMA per (m-tile, n-half).
__global__ void __launch_bounds__(kTI * kTJ) k_nn_midt(NnGrid g, const __nv_bfloat16* __restrict__ hin,
                                                     const __nv_bfloat16* __restrict__ wb,
                                                     const float* __restrict__ bias, float* __restrict__ z,
                                                     __nv_bfloat16* __restrict__ hout) {
  __shared__ __align__(128) uint4 pl[kRing][2][kPP];
  __shared__ uint32_t Ws[kTaps * kC * kC / 2];  // [tap][co][ci pair]
  __shared__ float Bs[kC];
  for (int q = threadIdx.x; q < kTaps * kC * kC / 2; q += blockDim.x) Ws[q] = reinterpret_cast<const uint32_t*>(wb)[q];
  for (int q = threadIdx.x; q < kC; q += blockDim.x) Bs[q] = bias[q];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, gq = lane >> 2, cq = lane & 3;
  const uint32_t* wl = Ws + gq * (kC / 2) + cq;  // this lane's B pairs: + tap * 128 (+4 high ci, +64 co + 8)
  const unsigned arow[2] = {a_row_addr(pl[0], w, 0, lane), a_row_addr(pl[0], w, 1, lane)};
  const unsigned sbase = (unsigned)__cvta_generic_to_shared(&pl[0][0][0]);
  const int tiles_i = (g.nx + kTI - 1) / kTI;
  const int64_t ntiles = (int64_t)tiles_i * ((g.ny + kTJ - 1) / kTJ);
  const int64_t plane = (int64_t)g.nx * g.ny * kC;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const TileGeo t = tile_geo(g, tile, tiles_i);
    PlaneCopy<2, 16> pc;
    pc.init(g, t);
    __syncthreads();
    for (int kq = 0; kq < 3; ++kq) {
      if (kq < g.nz) pc.issue(sbase + kq * kSlotBytes, hin, kq * plane);
      cp_async_commit();
    }
    cp_async_wait_one();
    __syncthreads();
    const int gj = t.j0 + w;
    for (int k = 0; k < g.nz; ++k) {
      if (k + 3 < g.nz) pc.issue(sbase + ((k + 3) % kRing) * kSlotBytes, hin, (int64_t)(k + 3) * plane);
      cp_async_commit();
      float d[2][2][4];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        d[mt][0][0] = d[mt][0][2] = Bs[2 * cq];
        d[mt][0][1] = d[mt][0][3] = Bs[2 * cq + 1];
        d[mt][1][0] = d[mt][1][2] = Bs[8 + 2 * cq];
        d[mt][1][1] = d[mt][1][3] = Bs[8 + 2 * cq + 1];
      }
      // planes of levels k-1, k, k+1 (a missing level contributes nothing)
      const unsigned sl[3] = {((k + kRing - 1) % kRing) * kSlotBytes, (k % kRing) * kSlotBytes,
                              ((k + 1) % kRing) * kSlotBytes};
      const bool has[3] = {k > 0, true, k + 1 < g.nz};
#pragma unroll
      for (int tp = 0; tp < kTaps; ++tp) {
        const int dk = tp / 9;
        if (!has[dk]) continue;
        const uint32_t b00 = wl[tp * 128], b01 = wl[tp * 128 + 4], b10 = wl[tp * 128 + 64], b11 = wl[tp * 128 + 68];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
          uint32_t a[4];
          ldmatrix_x4(a, arow[mt] + sl[dk] + tap_off(tp));
          mma_bf16_16816(d[mt][0], a, b00, b01);
          mma_bf16_16816(d[mt][1], a, b10, b11);
        }
      }
      if (gj < g.ny) {
        const int64_t prow = ((int64_t)k * g.ny + gj) * g.nx;
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
          for (int hf = 0; hf < 2; ++hf) {  // points gq (d[.][.][0..1]) and gq + 8 (d[.][.][2..3])
            const int gi = t.i0 + 16 * mt + gq + 8 * hf;
            if (gi >= g.nx) continue;
            const int64_t p = prow + gi;
            const float* v0 = &d[mt][0][2 * hf];
            const float* v1 = &d[mt][1][2 * hf];
            if (z) {
              *reinterpret_cast<float2*>(z + p * kC + 2 * cq) = make_float2(v0[0], v0[1]);
              *reinterpret_cast<float2*>(z + p * kC + 8 + 2 * cq) = make_float2(v1[0], v1[1]);
            }
            reinterpret_cast<__nv_bfloat162*>(hout + p * kC + 2 * cq)[0] =
                __floats2bfloat162_rn(gelu_f(v0[0]), gelu_f(v0[1]));
            reinterpret_cast<__nv_bfloat162*>(hout + p * kC + 8 + 2 * cq)[0] =
                __floats2bfloat162_rn(gelu_f(v1[0]), gelu_f(v1[1]));
          }
        }
      }
      cp_async_wait_one();
      __syncthreads();
    }
  }
  cp_async_wait_all();
}

// layer 4 on planes: 16 -> 1 as an m16n8k16 MMA whose B has one live column
// (output channel 0 = W4[tap][ci]).  out = y, or out = base + sigma * y.
__global__ void __launch_bounds__(kTI * kTJ) k_nn_l4t(NnGrid g, const __nv_bfloat16* __restrict__ hin, NnW w,
                                                    const float* base, const double* nrm2, float* out) {
  __shared__ __align__(128) uint4 pl[kRing][2][kPP];
  __shared__ uint32_t W4[kTaps * kC / 2];  // [tap][ci pair], BF16 (the values are BF16-rounded already)
  __shared__ float B4;
  for (int q = threadIdx.x; q < kTaps * kC / 2; q += blockDim.x) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(w.w4[2 * q], w.w4[2 * q + 1]);
    W4[q] = *reinterpret_cast<const uint32_t*>(&v);
  }
  if (threadIdx.x == 0) B4 = w.b4[0];
  float sigma = 1.f;
  if (nrm2) {
    const double v = *nrm2;
    sigma = (float)sqrt(v / (double)g.n);
  }
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, gq = lane >> 2, cq = lane & 3;
  const unsigned arow[2] = {a_row_addr(pl[0], wp, 0, lane), a_row_addr(pl[0], wp, 1, lane)};
  const unsigned sbase = (unsigned)__cvta_generic_to_shared(&pl[0][0][0]);
  const int tiles_i = (g.nx + kTI - 1) / kTI;
  const int64_t ntiles = (int64_t)tiles_i * ((g.ny + kTJ - 1) / kTJ);
  const int64_t plane = (int64_t)g.nx * g.ny * kC;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const TileGeo t = tile_geo(g, tile, tiles_i);
    PlaneCopy<2, 16> pc;
    pc.init(g, t);
    __syncthreads();
    for (int kq = 0; kq < 3; ++kq) {
      if (kq < g.nz) pc.issue(sbase + kq * kSlotBytes, hin, kq * plane);
      cp_async_commit();
    }
    cp_async_wait_one();
    __syncthreads();
    const int gj = t.j0 + wp;
    for (int k = 0; k < g.nz; ++k) {
      if (k + 3 < g.nz) pc.issue(sbase + ((k + 3) % kRing) * kSlotBytes, hin, (int64_t)(k + 3) * plane);
      cp_async_commit();
      float d[2][4];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) d[mt][0] = d[mt][1] = d[mt][2] = d[mt][3] = B4;
      const unsigned sl[3] = {((k + kRing - 1) % kRing) * kSlotBytes, (k % kRing) * kSlotBytes,
                              ((k + 1) % kRing) * kSlotBytes};
      const bool has[3] = {k > 0, true, k + 1 < g.nz};
#pragma unroll
      for (int tp = 0; tp < kTaps; ++tp) {
        const int dk = tp / 9;
        if (!has[dk]) continue;
        const uint32_t b0 = gq == 0 ? W4[tp * (kC / 2) + cq] : 0u;
        const uint32_t b1 = gq == 0 ? W4[tp * (kC / 2) + 4 + cq] : 0u;
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
          uint32_t a[4];
          ldmatrix_x4(a, arow[mt] + sl[dk] + tap_off(tp));
          mma_bf16_16816(d[mt], a, b0, b1);
        }
      }
      if (cq == 0 && gj < g.ny) {  // column 0 of D: points gq (d[.][0]) and gq + 8 (d[.][2])
        const int64_t prow = ((int64_t)k * g.ny + gj) * g.nx;
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
          for (int hf = 0; hf < 2; ++hf) {
            const int gi = t.i0 + 16 * mt + gq + 8 * hf;
            if (gi >= g.nx) continue;
            const int64_t p = prow + gi;
            const float y = d[mt][2 * hf];
            out[p] = base ? fmaf(sigma, y, base[p]) : y;
          }
        }
      }
      cp_async_wait_one();
      __syncthreads();
    }
  }
  cp_async_wait_all();
}

// ---- backward (FP32 on the CUDA cores) ---------------------------------------
// dz3[p][ci] = gelu'(z3[p][ci]) * sum_t W4[t][ci] dy[p - t]   (adjoint of layer 4)
__global__ void __launch_bounds__(256) k_nn_b4(NnGrid g, const float* __restrict__ dy, NnW w,
                                               const float* __restrict__ z3, float* __restrict__ dz3) {
  __shared__ float W[kTaps * kC];
  for (int q = threadIdx.x; q < kTaps * kC; q += blockDim.x) W[q] = w.w4[q];
  __syncthreads();
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < g.n; p += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(p % g.nx), j = (int)((p / g.nx) % g.ny), k = (int)(p / ((int64_t)g.nx * g.ny));
    float acc[kC];
#pragma unroll
    for (int c = 0; c < kC; ++c) acc[c] = 0.f;
    for (int t = 0; t < kTaps; ++t) {
      const int64_t q = nbr(g, i, j, k, kTaps - 1 - t);  // p - tap
      if (q < 0) continue;
      const float d = dy[q];
#pragma unroll
      for (int c = 0; c < kC; ++c) acc[c] = fmaf(W[t * kC + c], d, acc[c]);
    }
#pragma unroll
    for (int c = 0; c < kC; ++c) dz3[p * kC + c] = acc[c] * gelu_grad_f(z3[p * kC + c]);
  }
}

// dzo[p][ci] = gelu'(zo[p][ci]) * sum_t sum_co W[t][co][ci] dz[p - t][co]   (adjoint of a 16 -> 16 layer)
__global__ void __launch_bounds__(128) k_nn_bmid(NnGrid g, const float* __restrict__ dz, const float* __restrict__ wf,
                                                 const float* __restrict__ zo, float* __restrict__ dzo) {
  __shared__ float W[kTaps * kC * kC];
  for (int q = threadIdx.x; q < kTaps * kC * kC; q += blockDim.x) W[q] = wf[q];
  __syncthreads();
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < g.n; p += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(p % g.nx), j = (int)((p / g.nx) % g.ny), k = (int)(p / ((int64_t)g.nx * g.ny));
    float acc[kC];
#pragma unroll
    for (int c = 0; c < kC; ++c) acc[c] = 0.f;
    for (int t = 0; t < kTaps; ++t) {
      const int64_t q = nbr(g, i, j, k, kTaps - 1 - t);
      if (q < 0) continue;
      float d[kC];
#pragma unroll
      for (int c = 0; c < kC; c += 4) {
        const float4 v = *reinterpret_cast<const float4*>(dz + q * kC + c);
        d[c] = v.x, d[c + 1] = v.y, d[c + 2] = v.z, d[c + 3] = v.w;
      }
      const float* wt = W + t * kC * kC;
#pragma unroll
      for (int co = 0; co < kC; ++co)
#pragma unroll
        for (int ci = 0; ci < kC; ++ci) acc[ci] = fmaf(wt[co * kC + ci], d[co], acc[ci]);
    }
#pragma unroll
    for (int c = 0; c < kC; ++c) dzo[p * kC + c] = acc[c] * gelu_grad_f(zo[p * kC + c]);
  }
}

// Weight gradient of one layer, dW[co][ci][t] = sum_p dz[p][co] hin[p + t][ci]
// and db[co] = sum_p dz[p][co].  Block partials in FP64 (each thread owns
// output slots o = tid, tid + blockDim, ...; FP32 within a 32-point tile),
// written to part[block][slot]; k_nn_greduce sums them in block order.
template <int CI, int CO, typename HT>
__global__ void __launch_bounds__(256) k_nn_dw(NnGrid g, const float* __restrict__ dz, const HT* __restrict__ hin,
                                               double* __restrict__ part) {
  constexpr int NO = CO * CI * kTaps + CO;
  constexpr int TP = CI > 1 ? 16 : 32;  // points per tile: the staged neighbours stay under 48 KiB
  constexpr int PER = (NO + 255) / 256;
  __shared__ float sdz[TP][CO];
  __shared__ float sh[kTaps][TP][CI];
  double acc[PER];
#pragma unroll
  for (int u = 0; u < PER; ++u) acc[u] = 0.0;
  const int64_t ntile = (g.n + TP - 1) / TP;
  for (int64_t tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
    const int64_t p0 = tile * TP;
    __syncthreads();
    for (int q = threadIdx.x; q < TP * CO; q += blockDim.x) {
      const int pp = q / CO, c = q % CO;
      sdz[pp][c] = (p0 + pp < g.n) ? dz[(p0 + pp) * CO + c] : 0.f;
    }
    for (int q = threadIdx.x; q < kTaps * TP; q += blockDim.x) {
      const int t = q / TP, pp = q % TP;
      const int64_t p = p0 + pp;
      int64_t nb = -1;
      if (p < g.n) {
        const int i = (int)(p % g.nx), j = (int)((p / g.nx) % g.ny), k = (int)(p / ((int64_t)g.nx * g.ny));
        nb = nbr(g, i, j, k, t);
      }
#pragma unroll
      for (int c = 0; c < CI; ++c) {
        float v = 0.f;
        if (nb >= 0) {
          if constexpr (sizeof(HT) == 2)
            v = __bfloat162float(hin[nb * CI + c]);
          else
            v = (float)hin[nb * CI + c];
        }
        sh[t][pp][c] = v;
      }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int o = threadIdx.x + u * 256;
      if (o >= NO) continue;
      float s = 0.f;
      if (o < CO * CI * kTaps) {
        const int co = o / (CI * kTaps), rem = o % (CI * kTaps), ci = rem / kTaps, t = rem % kTaps;
        for (int pp = 0; pp < TP; ++pp) s = fmaf(sdz[pp][co], sh[t][pp][ci], s);
      } else {
        const int co = o - CO * CI * kTaps;
        for (int pp = 0; pp < TP; ++pp) s += sdz[pp][co];
      }
      acc[u] += (double)s;
    }
  }
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int o = threadIdx.x + u * 256;
    if (o < NO) part[(size_t)blockIdx.x * NO + o] = acc[u];
  }
}

// out[o] = sum_b part[b][o] in block order (deterministic)
__global__ void k_nn_greduce(const double* __restrict__ part, int nblocks, int no, double* __restrict__ out) {
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < no; o += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += part[(size_t)b * no + o];
    out[o] = s;
  }
}

// relative MSE over the interior of every crop (border points of each crop
// excluded in i and j): partials of sum (y - t)^2 and sum t^2
__device__ __forceinline__ bool in_mask(const NnGrid& g, int64_t p, int border) {
  const int i = (int)(p % g.nx), j = (int)((p / g.nx) % g.ny) % g.seg;
  return i >= border && i < g.nx - border && j >= border && j < g.seg - border;
}

__global__ void __launch_bounds__(256) k_nn_loss(NnGrid g, const float* __restrict__ y, const float* __restrict__ t,
                                                 int border, double* __restrict__ part) {
  double a = 0.0, b = 0.0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < g.n; p += (int64_t)gridDim.x * blockDim.x) {
    if (!in_mask(g, p, border)) continue;
    const double d = (double)y[p] - (double)t[p];
    a += d * d;
    b += (double)t[p] * (double)t[p];
  }
  __shared__ double sa[8], sb[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if (lane == 0) sa[warp] = a, sb[warp] = b;
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0.0, z = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) x += sa[w], z += sb[w];
    part[blockIdx.x * 2] = x;
    part[blockIdx.x * 2 + 1] = z;
  }
}

__global__ void k_nn_loss_fin(const double* __restrict__ part, int nblocks, double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double a = 0.0, b = 0.0;
  for (int q = 0; q < nblocks; ++q) a += part[2 * q], b += part[2 * q + 1];
  out[0] = b > 0.0 ? a / b : 0.0;  // loss
  out[1] = b;                       // sum t^2
}

// dy = 2 (y - t) / sum t^2 on the mask, 0 elsewhere
__global__ void __launch_bounds__(256) k_nn_dy(NnGrid g, const float* __restrict__ y, const float* __restrict__ t,
                                               int border, const double* __restrict__ lossv, float* __restrict__ dy) {
  const double tt = lossv[1];
  const float sc = tt > 0.0 ? (float)(2.0 / tt) : 0.f;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < g.n; p += (int64_t)gridDim.x * blockDim.x)
    dy[p] = in_mask(g, p, border) ? sc * (y[p] - t[p]) : 0.f;
}

// Operator-weighted loss on stacked training crops: u = mask (Ahat (y - t)),
// loss = ||u||^2 / ||mask Ahat t||^2 (with t = Ahat^-1 e1 the target of the
// stage, Ahat t = e1: the squared relative residual left after the stage).
// bands: the crops of the six scaled bands E, W, N, S, U, D at stride n.  On a
// crop, neighbours outside its columns, its segment of seg rows or the levels
// are absent (the mask keeps every term inside).
__global__ void __launch_bounds__(256) k_nn_oploss(NnGrid g, const float* __restrict__ y, const float* __restrict__ t,
                                                   const float* __restrict__ bands, int border, float* __restrict__ u,
                                                   double* __restrict__ part) {
  const int64_t plane = (int64_t)g.nx * g.ny, n = g.n;
  double a = 0.0, b = 0.0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    if (!in_mask(g, p, border)) {
      u[p] = 0.f;
      continue;
    }
    const int i = (int)(p % g.nx), jj = (int)((p / g.nx) % g.ny) % g.seg, k = (int)(p / plane);
    float ad = y[p] - t[p], at = t[p];
    auto add = [&](int b6, int64_t q) {
      const float c = bands[b6 * n + p];
      ad = fmaf(c, y[q] - t[q], ad);
      at = fmaf(c, t[q], at);
    };
    if (i + 1 < g.nx) add(0, p + 1);
    if (i > 0) add(1, p - 1);
    if (jj + 1 < g.seg) add(2, p + g.nx);
    if (jj > 0) add(3, p - g.nx);
    if (k + 1 < g.nz) add(4, p + plane);
    if (k > 0) add(5, p - plane);
    u[p] = ad;
    a += (double)ad * ad;
    b += (double)at * at;
  }
  __shared__ double sa[8], sb[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if (lane == 0) sa[warp] = a, sb[warp] = b;
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0.0, z = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) x += sa[w], z += sb[w];
    part[blockIdx.x * 2] = x;
    part[blockIdx.x * 2 + 1] = z;
  }
}

// dy = 2 Ahat^T u / ||mask Ahat t||^2: (Ahat^T u)[q] = u[q] + sum_b band_b[q - off_b] u[q - off_b]
__global__ void __launch_bounds__(256) k_nn_opdy(NnGrid g, const float* __restrict__ u,
                                                 const float* __restrict__ bands, const double* __restrict__ lossv,
                                                 float* __restrict__ dy) {
  const int64_t plane = (int64_t)g.nx * g.ny, n = g.n;
  const double den = lossv[1];
  const float sc = den > 0.0 ? (float)(2.0 / den) : 0.f;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(q % g.nx), jj = (int)((q / g.nx) % g.ny) % g.seg, k = (int)(q / plane);
    float v = u[q];
    if (i > 0) v = fmaf(bands[0 * n + q - 1], u[q - 1], v);
    if (i + 1 < g.nx) v = fmaf(bands[1 * n + q + 1], u[q + 1], v);
    if (jj > 0) v = fmaf(bands[2 * n + q - g.nx], u[q - g.nx], v);
    if (jj + 1 < g.seg) v = fmaf(bands[3 * n + q + g.nx], u[q + g.nx], v);
    if (k > 0) v = fmaf(bands[4 * n + q - plane], u[q - plane], v);
    if (k + 1 < g.nz) v = fmaf(bands[5 * n + q + plane], u[q + plane], v);
    dy[q] = sc * v;
  }
}

// Adam (Kingma & Ba) on the FP32 master parameters; lr, betas, eps and the
// bias corrections come from the host.
// global gradient norm (one block, fixed order) -> clipping factor min(1, clip / ||g||)
__global__ void k_nn_gclip(int np, const double* __restrict__ grad, double clip, double* __restrict__ factor) {
  __shared__ double sm[256];
  double s = 0.0;
  for (int q = threadIdx.x; q < np; q += blockDim.x) s += grad[q] * grad[q];
  sm[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)blockDim.x; ++w) t += sm[w];
    const double nrm = sqrt(t);
    *factor = (clip > 0.0 && nrm > clip) ? clip / nrm : 1.0;
  }
}

__global__ void k_nn_adam(int np, float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                          const double* __restrict__ grad, const double* __restrict__ gscale, float lr, float b1,
                          float b2, float eps, float c1, float c2) {
  const double gs = *gscale;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < np; q += gridDim.x * blockDim.x) {
    const float gq = (float)(grad[q] * gs);
    const float mq = b1 * m[q] + (1.f - b1) * gq;
    const float vq = b2 * v[q] + (1.f - b2) * gq * gq;
    m[q] = mq;
    v[q] = vq;
    w[q] -= lr * (mq / c1) / (sqrtf(vq / c2) + eps);
  }
}

// kernel-side weights from the FP32 master vector (bf16 rounding, re-layout)
__global__ void k_nn_refresh(const float* __restrict__ master, float* __restrict__ w1, float* __restrict__ b1,
                             __nv_bfloat16* __restrict__ w2b, float* __restrict__ w2f, float* __restrict__ b2,
                             __nv_bfloat16* __restrict__ w3b, float* __restrict__ w3f, float* __restrict__ b3,
                             float* __restrict__ w4, float* __restrict__ b4) {
  const int stride = gridDim.x * blockDim.x;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  auto rb = [](float x) { return __bfloat162float(__float2bfloat16_rn(x)); };
  for (int q = tid; q < kP1; q += stride) {  // master W1[co][0][t] -> w1[t][co]
    const int co = q / kTaps, t = q % kTaps;
    w1[t * kC + co] = rb(master[kOffW1 + q]);
  }
  for (int q = tid; q < kP2; q += stride) {  // master W[co][ci][t] -> [t][co][ci]
    const int co = q / (kC * kTaps), ci = (q / kTaps) % kC, t = q % kTaps;
    const int d = (t * kC + co) * kC + ci;
    const __nv_bfloat16 v2 = __float2bfloat16_rn(master[kOffW2 + q]);
    const __nv_bfloat16 v3 = __float2bfloat16_rn(master[kOffW3 + q]);
    w2b[d] = v2;
    w2f[d] = __bfloat162float(v2);
    w3b[d] = v3;
    w3f[d] = __bfloat162float(v3);
  }
  for (int q = tid; q < kP4; q += stride) {  // master W4[0][ci][t] -> w4[t][ci]
    const int ci = q / kTaps, t = q % kTaps;
    w4[t * kC + ci] = rb(master[kOffW4 + q]);
  }
  for (int q = tid; q < kC; q += stride) {
    b1[q] = rb(master[kOffB1 + q]);
    b2[q] = rb(master[kOffB2 + q]);
    b3[q] = rb(master[kOffB3 + q]);
  }
  if (tid == 0) b4[0] = rb(master[kOffB4]);
}

// training pair of one iterate x_k (Sec.-2 scaled system, FP64 in, FP32 out):
// r = D^-1 (b - A x_k) is the residual, e = x* - x_k the error; with
// z1 = T^-1 r and e1 = r - Ahat z1, the stage input is e1 / sigma and the
// target (e - z1) / sigma, sigma = rms(e1).  This kernel forms r (float) and
// e (float); the rest uses the solver's own T^-1 and residual kernels.
__global__ void __launch_bounds__(256) k_nn_pair_r(int64_t n, const double* __restrict__ A7, const double* __restrict__ b,
                                                  const double* __restrict__ xk, const double* __restrict__ xs,
                                                  const double* __restrict__ r, float* __restrict__ rs,
                                                  float* __restrict__ e) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    rs[p] = (float)(r[p] / A7[p]);
    e[p] = (float)(xs[p] - xk[p]);
  }
}

// in = e1 / sigma, target = (e - z1) / sigma with sigma = sqrt(nrm2 / n)
__global__ void __launch_bounds__(256) k_nn_pair_fin(int64_t n, const float* __restrict__ e1, const float* __restrict__ e,
                                                    const float* __restrict__ z1, const double* __restrict__ nrm2,
                                                    float* __restrict__ in, float* __restrict__ tg) {
  const double v = *nrm2;
  const float inv = v > 0.0 ? (float)(1.0 / sqrt(v / (double)n)) : 0.f;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    in[p] = e1[p] * inv;
    tg[p] = (e[p] - z1[p]) * inv;
  }
}

// Crops of (cy + 2h) x (cx + 2h) columns, all levels, from two fields, stacked
// along j: crop q starts at column (i0, j0) of the field (corners from the
// host), i wraps, rows outside [0, ny) are zero.
__global__ void __launch_bounds__(256) k_nn_crops(int nx, int ny, int nz, const float* __restrict__ fa,
                                                  const float* __restrict__ fb, int ncrop, int cx, int cy,
                                                  const int* __restrict__ corners, float* __restrict__ oa,
                                                  float* __restrict__ ob) {
  const int64_t per = (int64_t)cx * cy * nz;
  const int64_t total = per * ncrop;
  for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < total; o += (int64_t)gridDim.x * blockDim.x) {
    // output layout [k][q*cy + jj][ii] (crops stacked along j)
    const int ii = (int)(o % cx);
    const int64_t rowo = o / cx;
    const int jq = (int)(rowo % ((int64_t)cy * ncrop));
    const int k = (int)(rowo / ((int64_t)cy * ncrop));
    const int q = jq / cy, jj = jq % cy;
    const int i0 = corners[2 * q], j0 = corners[2 * q + 1];
    int i = (i0 + ii) % nx;
    if (i < 0) i += nx;
    const int j = j0 + jj;
    float va = 0.f, vb = 0.f;
    if (j >= 0 && j < ny) {
      const int64_t src = ((int64_t)k * ny + j) * nx + i;
      va = fa[src];
      vb = fb[src];
    }
    oa[o] = va;
    ob[o] = vb;
  }
}

}  // namespace hz

// ===========================================================================
// host side
// ===========================================================================
namespace hz {

static thread_local char g_nn_err[256] = "";

struct NnDev {
  float* master = nullptr;  // FP32 master parameters, flat layout
  float* m = nullptr;       // Adam moments
  float* v = nullptr;
  double* grad = nullptr;   // reduced gradient (FP64)
  float *w1 = nullptr, *b1 = nullptr, *w2f = nullptr, *b2 = nullptr, *w3f = nullptr, *b3 = nullptr, *w4 = nullptr,
        *b4 = nullptr;
  __nv_bfloat16 *w2b = nullptr, *w3b = nullptr;
  int64_t cap = 0;
  __nv_bfloat16 *h1 = nullptr, *h2 = nullptr, *h3 = nullptr;
  float *z1 = nullptr, *z2 = nullptr, *z3 = nullptr, *dza = nullptr, *dzb = nullptr, *y = nullptr, *dy = nullptr;
  int train_cap = 0;  // 1 if the training buffers exist for cap points
  double* part = nullptr;
  int64_t part_cap = 0;
  double* lossv = nullptr;
  double* lossh = nullptr;
  int* err = nullptr;       // device error word of the tensor-core kernels (bit 0: a bounded wait gave up)
  int step = 0;
};

}  // namespace hz

struct hz_nn_s {
  hz::NnDev d;
  cudaStream_t stream = nullptr;
  int sms = 0;
};

namespace hz {

#define NN_CK(call)                                                                               \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess) {                                                                      \
      snprintf(g_nn_err, sizeof(g_nn_err), "%s at hz_nn.cu:%d: %s", cudaGetErrorName(e_), __LINE__, #call); \
      return e_ == cudaErrorMemoryAllocation ? HZ_ERR_OOM : HZ_ERR_CUDA;                          \
    }                                                                                             \
  } while (0)

// the tensor-core kernels' error word: a bounded wait that gave up (reset when read)
static int nn_check_err(hz_nn_s* nn) {
  int e = 0;
  NN_CK(cudaMemcpy(&e, nn->d.err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e) {
    NN_CK(cudaMemset(nn->d.err, 0, sizeof(int)));
    snprintf(g_nn_err, sizeof(g_nn_err), "tensor-core convolution: a completion wait exceeded its limit");
    return HZ_ERR_TIMEOUT;
  }
  return HZ_OK;
}

static NnW nn_w(const NnDev& d) {
  return NnW{d.w1, d.b1, d.w2b, d.w2f, d.b2, d.w3b, d.w3f, d.b3, d.w4, d.b4};
}

static int nn_grid(const hz_nn_s* nn, int64_t n, int block) {
  int64_t g = (int64_t)nn->sms * 8;
  const int64_t need = (n + block - 1) / block;
  if (g > need) g = need;
  return g < 1 ? 1 : (int)g;
}

static int nn_refresh(hz_nn_s* nn) {
  NnDev& d = nn->d;
  k_nn_refresh<<<32, 256, 0, nn->stream>>>(d.master, d.w1, d.b1, d.w2b, d.w2f, d.b2, d.w3b, d.w3f, d.b3, d.w4, d.b4);
  NN_CK(cudaGetLastError());
  return HZ_OK;
}

static int nn_reserve(hz_nn_s* nn, int64_t n, bool train) {
  NnDev& d = nn->d;
  if (n <= d.cap && (!train || d.train_cap)) return HZ_OK;
  NN_CK(cudaStreamSynchronize(nn->stream));
  for (void* p : {(void*)d.h1, (void*)d.h2, (void*)d.h3, (void*)d.z1, (void*)d.z2, (void*)d.z3, (void*)d.dza,
                  (void*)d.dzb, (void*)d.y, (void*)d.dy})
    if (p) cudaFree(p);
  d.h1 = d.h2 = d.h3 = nullptr;
  d.z1 = d.z2 = d.z3 = d.dza = d.dzb = d.y = d.dy = nullptr;
  const int64_t c = n > d.cap ? n : d.cap;
  NN_CK(cudaMalloc(&d.h1, sizeof(__nv_bfloat16) * kC * c));
  NN_CK(cudaMalloc(&d.h2, sizeof(__nv_bfloat16) * kC * c));
  d.train_cap = 0;
  if (train) {
    NN_CK(cudaMalloc(&d.h3, sizeof(__nv_bfloat16) * kC * c));
    NN_CK(cudaMalloc(&d.z1, sizeof(float) * kC * c));
    NN_CK(cudaMalloc(&d.z2, sizeof(float) * kC * c));
    NN_CK(cudaMalloc(&d.z3, sizeof(float) * kC * c));
    NN_CK(cudaMalloc(&d.dza, sizeof(float) * kC * c));
    NN_CK(cudaMalloc(&d.dzb, sizeof(float) * kC * c));
    NN_CK(cudaMalloc(&d.y, sizeof(float) * c));
    NN_CK(cudaMalloc(&d.dy, sizeof(float) * c));
    d.train_cap = 1;
  }
  d.cap = c;
  return HZ_OK;
}

// forward pass; train: keep z1..z3 and h1..h3 for the backward pass.
// x scaled by 1/sigma (sigma from *scale_nrm2) when scale_nrm2 is given.
// Output: out = y, or out = base + sigma * y when base is given.
static int nn_forward(hz_nn_s* nn, const NnGrid& g, const float* x, const double* scale_nrm2, bool train,
                      const float* base, float* out) {
  NnDev& d = nn->d;
  const NnW w = nn_w(d);
  cudaStream_t s = nn->stream;
  __nv_bfloat16* h3 = train ? d.h3 : d.h1;
  if (g.seg == g.ny || g.seg % kTJ == 0) {  // plane-tiled kernels: no tile straddles a crop seam
    const int64_t tiles = (int64_t)((g.nx + kTI - 1) / kTI) * ((g.ny + kTJ - 1) / kTJ);
    const int gt = (int)std::min<int64_t>(tiles, (int64_t)nn->sms * 4);
    k_nn_l1t<<<gt, kTI * kTJ, 0, s>>>(g, x, scale_nrm2, w, train ? d.z1 : nullptr, d.h1);
    if (nn_tc_ok(g)) {  // 16 -> 16 and 16 -> 1 on tcgen05 (rows of 128 points)
      NN_CK(nn_tc_mid(g, d.h1, d.w2b, d.b2, train ? d.z2 : nullptr, d.h2, d.err, nn->sms, s));
      NN_CK(nn_tc_mid(g, d.h2, d.w3b, d.b3, train ? d.z3 : nullptr, h3, d.err, nn->sms, s));
      NN_CK(nn_tc_l4(g, h3, d.w4, d.b4, base, base ? scale_nrm2 : nullptr, out, d.err, nn->sms, s));
      return HZ_OK;
    }
    k_nn_midt<<<gt, kTI * kTJ, 0, s>>>(g, d.h1, d.w2b, d.b2, train ? d.z2 : nullptr, d.h2);
    k_nn_midt<<<gt, kTI * kTJ, 0, s>>>(g, d.h2, d.w3b, d.b3, train ? d.z3 : nullptr, h3);
    k_nn_l4t<<<gt, kTI * kTJ, 0, s>>>(g, h3, w, base, base ? scale_nrm2 : nullptr, out);
    NN_CK(cudaGetLastError());
    return HZ_OK;
  }
  k_nn_l1<<<nn_grid(nn, g.n, 256), 256, 0, s>>>(g, x, scale_nrm2, 1.f, w, train ? d.z1 : nullptr, d.h1);
  const int64_t tiles = (int64_t)((g.nx + 15) / 16) * g.ny * g.nz;
  const int gm = (int)std::min<int64_t>((tiles + 3) / 4, (int64_t)nn->sms * 16);
  k_nn_mid<<<gm, 128, 0, s>>>(g, d.h1, d.w2b, d.b2, train ? d.z2 : nullptr, d.h2);
  k_nn_mid<<<gm, 128, 0, s>>>(g, d.h2, d.w3b, d.b3, train ? d.z3 : nullptr, h3);
  k_nn_l4<<<nn_grid(nn, g.n, 256), 256, 0, s>>>(g, h3, w, base, base ? scale_nrm2 : nullptr, out);
  NN_CK(cudaGetLastError());
  return HZ_OK;
}

template <int CI, int CO, typename HT>
static int nn_dw(hz_nn_s* nn, const NnGrid& g, const float* dz, const HT* hin, double* dst) {
  NnDev& d = nn->d;
  constexpr int NO = CO * CI * kTaps + CO;
  const int64_t ntile = (g.n + 31) / 32;
  const int grid = (int)std::min<int64_t>(ntile, (int64_t)nn->sms * 4);
  if (d.part_cap < (int64_t)grid * NO) {
    NN_CK(cudaStreamSynchronize(nn->stream));
    if (d.part) cudaFree(d.part);
    NN_CK(cudaMalloc(&d.part, sizeof(double) * (size_t)grid * NO));
    d.part_cap = (int64_t)grid * NO;
  }
  k_nn_dw<CI, CO, HT><<<grid, 256, 0, nn->stream>>>(g, dz, hin, d.part);
  k_nn_greduce<<<(NO + 255) / 256, 256, 0, nn->stream>>>(d.part, grid, NO, dst);
  NN_CK(cudaGetLastError());
  return HZ_OK;
}

// forward + masked loss + backward: d.grad, d.lossv.  bands == nullptr: the
// relative MSE of the output against t; else the operator-weighted loss with
// the crops' scaled bands (border then bounds the residual's mask)
static int nn_gradient(hz_nn_s* nn, const NnGrid& g, int border, const float* x, const float* t,
                       const float* bands = nullptr) {
  NnDev& d = nn->d;
  cudaStream_t s = nn->stream;
  int st = nn_reserve(nn, g.n, true);
  if (st != HZ_OK) return st;
  if ((st = nn_forward(nn, g, x, nullptr, true, nullptr, d.y)) != HZ_OK) return st;
  const int gl = nn_grid(nn, g.n, 256);
  if (d.part_cap < 2 * gl) {
    NN_CK(cudaStreamSynchronize(s));
    if (d.part) cudaFree(d.part);
    NN_CK(cudaMalloc(&d.part, sizeof(double) * 2 * gl));
    d.part_cap = 2 * gl;
  }
  if (bands) {
    k_nn_oploss<<<gl, 256, 0, s>>>(g, d.y, t, bands, border, d.dzb, d.part);  // u in the dz2 scratch
    k_nn_loss_fin<<<1, 32, 0, s>>>(d.part, gl, d.lossv);
    k_nn_opdy<<<gl, 256, 0, s>>>(g, d.dzb, bands, d.lossv, d.dy);
  } else {
    k_nn_loss<<<gl, 256, 0, s>>>(g, d.y, t, border, d.part);
    k_nn_loss_fin<<<1, 32, 0, s>>>(d.part, gl, d.lossv);
    k_nn_dy<<<gl, 256, 0, s>>>(g, d.y, t, border, d.lossv, d.dy);
  }
  const NnW w = nn_w(d);
  // layer 4
  k_nn_b4<<<gl, 256, 0, s>>>(g, d.dy, w, d.z3, d.dza);  // dz3
  if ((st = nn_dw<kC, 1, __nv_bfloat16>(nn, g, d.dy, d.h3, d.grad + kOffW4)) != HZ_OK) return st;
  // layer 3
  k_nn_bmid<<<nn_grid(nn, g.n, 128), 128, 0, s>>>(g, d.dza, d.w3f, d.z2, d.dzb);  // dz2
  if ((st = nn_dw<kC, kC, __nv_bfloat16>(nn, g, d.dza, d.h2, d.grad + kOffW3)) != HZ_OK) return st;
  // layer 2
  k_nn_bmid<<<nn_grid(nn, g.n, 128), 128, 0, s>>>(g, d.dzb, d.w2f, d.z1, d.dza);  // dz1
  if ((st = nn_dw<kC, kC, __nv_bfloat16>(nn, g, d.dzb, d.h1, d.grad + kOffW2)) != HZ_OK) return st;
  // layer 1
  if ((st = nn_dw<1, kC, float>(nn, g, d.dza, x, d.grad + kOffW1)) != HZ_OK) return st;
  NN_CK(cudaGetLastError());
  return HZ_OK;
}

// the learned stage inside the flexible solver (called by the engine):
// z <- z + sigma * NN(e1 / sigma), sigma = sqrt(nrm2 / n)
int nn_stage_apply(hz_nn_s* nn, const Grid& gr, const float* e1, const double* nrm2, float* z, cudaStream_t s) {
  NnGrid g{gr.nx, gr.ny, gr.nz, gr.ny, 1, gr.n};
  cudaStream_t keep = nn->stream;
  nn->stream = s;
  int st = nn_reserve(nn, g.n, false);
  if (st == HZ_OK) st = nn_forward(nn, g, e1, nrm2, false, z, z);
  nn->stream = keep;
  return st;
}

int nn_stage_status(hz_nn_s* nn, cudaStream_t s) {
  NN_CK(cudaStreamSynchronize(s));
  return nn_check_err(nn);
}

cudaError_t nn_pair_launch(int64_t n, const double* A7, const double* b, const double* xk, const double* xs,
                           const double* r, float* rs, float* e, const float* e1, const float* z1, const double* nrm2,
                           float* in, float* tg, int stage, cudaStream_t s) {
  const int grid = (int)std::min<int64_t>((n + 255) / 256, 8192);
  if (stage == 0)
    k_nn_pair_r<<<grid, 256, 0, s>>>(n, A7, b, xk, xs, r, rs, e);
  else
    k_nn_pair_fin<<<grid, 256, 0, s>>>(n, e1, e, z1, nrm2, in, tg);
  return cudaGetLastError();
}

}  // namespace hz

using namespace hz;

static bool nn_is_dev(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

extern "C" {

int hz_nn_num_params(void) { return kNParams; }

const char* hz_nn_last_error(void) { return g_nn_err; }

int hz_nn_create(void* stream, hz_nn* out) {
  if (!out) return HZ_ERR_INVALID;
  *out = nullptr;
  hz_nn_s* nn = new hz_nn_s();
  nn->stream = (cudaStream_t)stream;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nn->sms, cudaDevAttrMultiProcessorCount, dev);
  NnDev& d = nn->d;
  auto fail = [&](int st) {
    hz_nn_destroy(nn);
    return st;
  };
  if (cudaMalloc(&d.master, sizeof(float) * kNParams) != cudaSuccess) return fail(HZ_ERR_OOM);
  if (cudaMalloc(&d.err, sizeof(int)) != cudaSuccess) return fail(HZ_ERR_OOM);
  if (cudaMemset(d.err, 0, sizeof(int)) != cudaSuccess) return fail(HZ_ERR_CUDA);
  if (cudaMalloc(&d.m, sizeof(float) * kNParams) != cudaSuccess) return fail(HZ_ERR_OOM);
  if (cudaMalloc(&d.v, sizeof(float) * kNParams) != cudaSuccess) return fail(HZ_ERR_OOM);
  if (cudaMalloc(&d.grad, sizeof(double) * kNParams) != cudaSuccess) return fail(HZ_ERR_OOM);
  if (cudaMalloc(&d.w1, sizeof(float) * (kP1 + kC + 2 * (kP2 + kC) + kP4 + 1)) != cudaSuccess) return fail(HZ_ERR_OOM);
  d.b1 = d.w1 + kP1;
  d.w2f = d.b1 + kC;
  d.b2 = d.w2f + kP2;
  d.w3f = d.b2 + kC;
  d.b3 = d.w3f + kP2;
  d.w4 = d.b3 + kC;
  d.b4 = d.w4 + kP4;
  if (cudaMalloc(&d.w2b, sizeof(__nv_bfloat16) * 2 * kP2) != cudaSuccess) return fail(HZ_ERR_OOM);
  d.w3b = d.w2b + kP2;
  if (cudaMalloc(&d.lossv, sizeof(double) * 4) != cudaSuccess) return fail(HZ_ERR_OOM);
  if (cudaMallocHost(&d.lossh, sizeof(double) * 2) != cudaSuccess) return fail(HZ_ERR_OOM);
  cudaMemsetAsync(d.master, 0, sizeof(float) * kNParams, nn->stream);
  cudaMemsetAsync(d.m, 0, sizeof(float) * kNParams, nn->stream);
  cudaMemsetAsync(d.v, 0, sizeof(float) * kNParams, nn->stream);
  if (nn_refresh(nn) != HZ_OK) return fail(HZ_ERR_CUDA);
  if (cudaStreamSynchronize(nn->stream) != cudaSuccess) return fail(HZ_ERR_CUDA);
  *out = nn;
  return HZ_OK;
}

int hz_nn_destroy(hz_nn nn) {
  if (!nn) return HZ_OK;
  cudaStreamSynchronize(nn->stream);
  NnDev& d = nn->d;
  for (void* p : {(void*)d.master, (void*)d.m, (void*)d.v, (void*)d.grad, (void*)d.w1, (void*)d.w2b, (void*)d.lossv,
                  (void*)d.h1, (void*)d.h2, (void*)d.h3, (void*)d.z1, (void*)d.z2, (void*)d.z3, (void*)d.dza,
                  (void*)d.dzb, (void*)d.y, (void*)d.dy, (void*)d.part, (void*)d.err})
    if (p) cudaFree(p);
  if (d.lossh) cudaFreeHost(d.lossh);
  delete nn;
  return HZ_OK;
}

int hz_nn_set_params(hz_nn nn, const float* params) {
  if (!nn || !params) return HZ_ERR_INVALID;
  NnDev& d = nn->d;
  NN_CK(cudaMemcpyAsync(d.master, params, sizeof(float) * kNParams,
                        nn_is_dev(params) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, nn->stream));
  NN_CK(cudaMemsetAsync(d.m, 0, sizeof(float) * kNParams, nn->stream));
  NN_CK(cudaMemsetAsync(d.v, 0, sizeof(float) * kNParams, nn->stream));
  d.step = 0;
  int st = nn_refresh(nn);
  if (st != HZ_OK) return st;
  NN_CK(cudaStreamSynchronize(nn->stream));
  return HZ_OK;
}

int hz_nn_get_params(hz_nn nn, float* out) {
  if (!nn || !out) return HZ_ERR_INVALID;
  NN_CK(cudaMemcpyAsync(out, nn->d.master, sizeof(float) * kNParams,
                        nn_is_dev(out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, nn->stream));
  NN_CK(cudaStreamSynchronize(nn->stream));
  return HZ_OK;
}

int hz_nn_forward(hz_nn nn, int nx, int ny, int nz, int seg_ny, int periodic, const float* x, float* y, float* zout) {
  if (!nn || !x || !y || nx < 1 || ny < 1 || nz < 1 || seg_ny < 1 || ny % seg_ny) return HZ_ERR_INVALID;
  NnGrid g{nx, ny, nz, seg_ny, periodic ? 1 : 0, (int64_t)nx * ny * nz};
  int st = nn_reserve(nn, g.n, zout != nullptr);
  if (st != HZ_OK) return st;
  st = nn_forward(nn, g, x, nullptr, zout != nullptr, nullptr, y);
  if (st != HZ_OK) return st;
  if (zout) {  // pre-activations z1, z2, z3 (FP32, [3][n][16])
    NN_CK(cudaMemcpyAsync(zout, nn->d.z1, sizeof(float) * kC * g.n, cudaMemcpyDeviceToDevice, nn->stream));
    NN_CK(cudaMemcpyAsync(zout + kC * g.n, nn->d.z2, sizeof(float) * kC * g.n, cudaMemcpyDeviceToDevice, nn->stream));
    NN_CK(cudaMemcpyAsync(zout + 2 * kC * g.n, nn->d.z3, sizeof(float) * kC * g.n, cudaMemcpyDeviceToDevice,
                          nn->stream));
  }
  NN_CK(cudaStreamSynchronize(nn->stream));
  return nn_check_err(nn);
}

int hz_nn_gradient(hz_nn nn, int nx, int ny, int nz, int seg_ny, int periodic, int border, const float* x,
                   const float* t, double* grad, double* loss) {
  if (!nn || !x || !t || nx < 1 || ny < 1 || nz < 1 || seg_ny < 1 || ny % seg_ny || border < 0) return HZ_ERR_INVALID;
  NnGrid g{nx, ny, nz, seg_ny, periodic ? 1 : 0, (int64_t)nx * ny * nz};
  int st = nn_gradient(nn, g, border, x, t);
  if (st != HZ_OK) return st;
  if (grad)
    NN_CK(cudaMemcpyAsync(grad, nn->d.grad, sizeof(double) * kNParams,
                          nn_is_dev(grad) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, nn->stream));
  NN_CK(cudaMemcpyAsync(nn->d.lossh, nn->d.lossv, sizeof(double) * 2, cudaMemcpyDeviceToHost, nn->stream));
  NN_CK(cudaStreamSynchronize(nn->stream));
  if (loss) *loss = nn->d.lossh[0];
  return HZ_OK;
}

}  // extern "C"

// one Adam step on the gradient of the loss (nn_gradient's choice by bands)
static int nn_train_step(hz_nn nn, const NnGrid& g, int border, const float* x, const float* t, const float* bands,
                         double lr, double clip, double* loss) {
  int st = nn_gradient(nn, g, border, x, t, bands);
  if (st != HZ_OK) return st;
  NnDev& d = nn->d;
  d.step += 1;
  const double b1 = 0.9, b2 = 0.999;
  const float c1 = (float)(1.0 - std::pow(b1, d.step)), c2 = (float)(1.0 - std::pow(b2, d.step));
  k_nn_gclip<<<1, 256, 0, nn->stream>>>(kNParams, d.grad, clip, d.lossv + 2);
  k_nn_adam<<<(kNParams + 255) / 256, 256, 0, nn->stream>>>(kNParams, d.master, d.m, d.v, d.grad, d.lossv + 2, (float)lr,
                                                             (float)b1, (float)b2, 1e-8f, c1, c2);
  NN_CK(cudaGetLastError());
  if ((st = nn_refresh(nn)) != HZ_OK) return st;
  if (loss) {
    NN_CK(cudaMemcpyAsync(d.lossh, d.lossv, sizeof(double) * 2, cudaMemcpyDeviceToHost, nn->stream));
    NN_CK(cudaStreamSynchronize(nn->stream));
    *loss = d.lossh[0];
  }
  return HZ_OK;
}

extern "C" {

int hz_nn_train_step(hz_nn nn, int nx, int ny, int nz, int seg_ny, int periodic, int border, const float* x,
                     const float* t, double lr, double clip, double* loss) {
  if (!nn || !x || !t || nx < 1 || ny < 1 || nz < 1 || seg_ny < 1 || ny % seg_ny || border < 0 || !(lr > 0))
    return HZ_ERR_INVALID;
  NnGrid g{nx, ny, nz, seg_ny, periodic ? 1 : 0, (int64_t)nx * ny * nz};
  return nn_train_step(nn, g, border, x, t, nullptr, lr, clip, loss);
}

int hz_nn_gradient_op(hz_nn nn, int nx, int ny, int nz, int seg_ny, int border, const float* x, const float* t,
                      const float* bands, double* grad, double* loss) {
  if (!nn || !x || !t || !bands || !grad || nx < 1 || ny < 1 || nz < 1 || seg_ny < 1 || ny % seg_ny || border < 1)
    return HZ_ERR_INVALID;
  NnGrid g{nx, ny, nz, seg_ny, 0, (int64_t)nx * ny * nz};
  int st = nn_gradient(nn, g, border, x, t, bands);
  if (st != HZ_OK) return st;
  NnDev& d = nn->d;
  NN_CK(cudaMemcpyAsync(d.lossh, d.lossv, sizeof(double) * 2, cudaMemcpyDeviceToHost, nn->stream));
  NN_CK(cudaMemcpyAsync(grad, d.grad, sizeof(double) * kNParams, cudaMemcpyDefault, nn->stream));
  NN_CK(cudaStreamSynchronize(nn->stream));
  if (loss) *loss = d.lossh[0];
  return HZ_OK;
}

int hz_nn_crops(int nx, int ny, int nz, const float* fa, const float* fb, int ncrop, int cx, int cy,
                const int* corners, float* oa, float* ob, void* stream) {
  if (nx < 1 || ny < 1 || nz < 1 || !fa || !fb || ncrop < 1 || cx < 1 || cy < 1 || !corners || !oa || !ob)
    return HZ_ERR_INVALID;
  for (int q = 0; q < ncrop; ++q)
    if (corners[2 * q + 1] < -cy || corners[2 * q + 1] > ny) return HZ_ERR_INVALID;
  int* dc = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  NN_CK(cudaMallocAsync((void**)&dc, sizeof(int) * 2 * ncrop, s));
  NN_CK(cudaMemcpyAsync(dc, corners, sizeof(int) * 2 * ncrop, cudaMemcpyHostToDevice, s));
  const int64_t total = (int64_t)cx * cy * nz * ncrop;
  k_nn_crops<<<(int)std::min<int64_t>((total + 255) / 256, 8192), 256, 0, s>>>(nx, ny, nz, fa, fb, ncrop, cx, cy, dc,
                                                                               oa, ob);
  NN_CK(cudaGetLastError());
  NN_CK(cudaFreeAsync(dc, s));
  NN_CK(cudaStreamSynchronize(s));
  return HZ_OK;
}

int hz_nn_save(hz_nn nn, const char* path) {
  if (!nn || !path) return HZ_ERR_INVALID;
  std::vector<float> buf(3 * kNParams);
  NN_CK(cudaMemcpyAsync(buf.data(), nn->d.master, sizeof(float) * kNParams, cudaMemcpyDeviceToHost, nn->stream));
  NN_CK(cudaMemcpyAsync(buf.data() + kNParams, nn->d.m, sizeof(float) * kNParams, cudaMemcpyDeviceToHost, nn->stream));
  NN_CK(cudaMemcpyAsync(buf.data() + 2 * kNParams, nn->d.v, sizeof(float) * kNParams, cudaMemcpyDeviceToHost,
                        nn->stream));
  NN_CK(cudaStreamSynchronize(nn->stream));
  FILE* f = fopen(path, "wb");
  if (!f) return HZ_ERR_INVALID;
  const char magic[8] = {'H', 'Z', 'N', 'N', '0', '0', '0', '1'};
  const int32_t hdr[2] = {kNParams, nn->d.step};
  bool ok = fwrite(magic, 1, 8, f) == 8 && fwrite(hdr, sizeof(int32_t), 2, f) == 2 &&
            fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
  ok = (fclose(f) == 0) && ok;
  return ok ? HZ_OK : HZ_ERR_INVALID;
}

int hz_nn_load(hz_nn nn, const char* path) {
  if (!nn || !path) return HZ_ERR_INVALID;
  FILE* f = fopen(path, "rb");
  if (!f) return HZ_ERR_INVALID;
  char magic[8];
  int32_t hdr[2];
  std::vector<float> buf(3 * kNParams);
  bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, "HZNN0001", 8) == 0 && fread(hdr, sizeof(int32_t), 2, f) == 2 &&
            hdr[0] == kNParams && fread(buf.data(), sizeof(float), buf.size(), f) == buf.size();
  fclose(f);
  if (!ok) return HZ_ERR_INVALID;
  NnDev& d = nn->d;
  NN_CK(cudaMemcpyAsync(d.master, buf.data(), sizeof(float) * kNParams, cudaMemcpyHostToDevice, nn->stream));
  NN_CK(cudaMemcpyAsync(d.m, buf.data() + kNParams, sizeof(float) * kNParams, cudaMemcpyHostToDevice, nn->stream));
  NN_CK(cudaMemcpyAsync(d.v, buf.data() + 2 * kNParams, sizeof(float) * kNParams, cudaMemcpyHostToDevice, nn->stream));
  d.step = hdr[1];
  int st = nn_refresh(nn);
  if (st != HZ_OK) return st;
  NN_CK(cudaStreamSynchronize(nn->stream));
  return HZ_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Training on one system (pairs, crops and Adam steps; see include/hz.h).
namespace {

// SplitMix64 finaliser (Steele, Lea and Flood 2014): a counter-based stream
// keyed by (seed, stream, counter); uniform in [0, 1) from the top 53 bits
uint64_t sm64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
double draw(uint64_t seed, uint64_t stream, uint64_t counter) {
  const uint64_t h = sm64(sm64(sm64(seed) ^ stream) ^ counter);
  return (double)(h >> 11) * (1.0 / 9007199254740992.0);
}

constexpr int kHalo = 4;  // receptive field of four 3x3x3 layers

struct TrainBufs {
  std::vector<void*> ptrs;
  ~TrainBufs() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <typename T>
  T* get(int64_t count) {
    void* p = nullptr;
    if (cudaMalloc(&p, sizeof(T) * (size_t)count) != cudaSuccess) return nullptr;
    ptrs.push_back(p);
    return (T*)p;
  }
};

}  // namespace

extern "C" {

void hz_nn_train_defaults(hz_nn_train_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->steps = 40;
  p->batch = 16;
  p->crop = 64;
  p->n_iterates = 6;
  for (int q = 0; q < 6; ++q) p->iterates[q] = 1 << q;
  p->xstar_tol = 1e-11;
  p->lr = 3e-4;
  p->clip = 1.0;
  p->seed = 7;
  p->stream = 0;
  p->loss = 1;
}

int hz_nn_train(hz_nn nn, hz_op op, const double* b, const hz_nn_train_params* pp, double* losses) {
  if (!nn || !op || !b || !pp) return HZ_ERR_INVALID;
  const hz_nn_train_params p = *pp;
  if (p.steps < 0 || p.batch < 1 || p.crop < 1 || p.n_iterates < 1 || p.n_iterates > 16 || !(p.lr > 0.0) ||
      !(p.xstar_tol > 0.0) || (p.loss != 0 && p.loss != 1))
    return HZ_ERR_INVALID;
  for (int q = 0; q < p.n_iterates; ++q)
    if (p.iterates[q] < 1) return HZ_ERR_INVALID;
  int nx = 0, ny = 0, nz = 0;
  int st = hz_op_dims(op, &nx, &ny, &nz);
  if (st != HZ_OK) return st;
  const int cx = p.crop + 2 * kHalo, cy = cx;
  if (cx > nx || p.crop >= ny) return HZ_ERR_INVALID;
  const int64_t n = (int64_t)nx * ny * nz;
  TrainBufs bufs;
  double* xs = bufs.get<double>(n);
  double* xk = bufs.get<double>(n);
  float* pin = bufs.get<float>(n * p.n_iterates);
  float* ptg = bufs.get<float>(n * p.n_iterates);
  const int64_t cn = (int64_t)p.batch * cx * cy * nz;
  float* bin = bufs.get<float>(cn);
  float* btg = bufs.get<float>(cn);
  // the operator-weighted loss also needs the scaled bands on every crop
  const bool opl = p.loss == 1;
  float* b6 = opl ? bufs.get<float>(6 * n) : nullptr;
  float* bcr = opl ? bufs.get<float>(6 * cn) : nullptr;
  if (!xs || !xk || !pin || !ptg || !bin || !btg || (opl && (!b6 || !bcr))) {
    snprintf(g_nn_err, sizeof(g_nn_err), "hz_nn_train: device allocation failed");
    return HZ_ERR_OOM;
  }
  if (opl && (st = hz_op_export(op, 0, HZ_PREC_FP32, b6)) != HZ_OK) return st;
  // 1. the exact solution
  hz_solve_params sp;
  hz_default_params(&sp);
  sp.mode = HZ_MODE_FP64;
  sp.tol = p.xstar_tol;
  hz_solve_info info;
  st = hz_solve(op, b, nullptr, xs, &sp, &info);
  if (st != HZ_OK && st != HZ_ERR_NOT_CONVERGED) return st;
  // 2. iterates of the plain mixed solver and their pairs
  int npairs = 0;
  for (int q = 0; q < p.n_iterates; ++q) {
    hz_default_params(&sp);
    sp.max_outer = 1;
    sp.max_inner = p.iterates[q];
    sp.inner_tol = 1e-12;
    st = hz_solve(op, b, nullptr, xk, &sp, &info);
    if (st != HZ_OK && st != HZ_ERR_NOT_CONVERGED) return st;
    if (info.inner_iters < 1) continue;
    double sigma = 0.0;
    st = hz_nn_make_pair(op, b, xk, xs, pin + npairs * n, ptg + npairs * n, &sigma);
    if (st != HZ_OK) return st;
    if (!(sigma > 0.0) || !std::isfinite(sigma)) continue;
    ++npairs;
  }
  if (npairs == 0) {
    snprintf(g_nn_err, sizeof(g_nn_err), "hz_nn_train: no usable training pair (the system converged at once)");
    return HZ_ERR_INVALID;
  }
  // 3. Adam steps on random crops of random pairs
  std::vector<int> corners(2 * p.batch);
  uint64_t ctr = 0;
  const int jspan = ny - p.crop > 1 ? ny - p.crop : 1;
  for (int it = 0; it < p.steps; ++it) {
    int pi = (int)(draw(p.seed, 2 * p.stream, ctr++) * npairs);
    if (pi >= npairs) pi = npairs - 1;
    for (int q = 0; q < p.batch; ++q) {
      int i0 = (int)(draw(p.seed, 2 * p.stream + 1, ctr++) * nx);
      int j0 = (int)(draw(p.seed, 2 * p.stream + 1, ctr++) * jspan);
      if (i0 >= nx) i0 = nx - 1;
      if (j0 >= jspan) j0 = jspan - 1;
      corners[2 * q] = i0 - kHalo;
      corners[2 * q + 1] = j0 - kHalo;
    }
    st = hz_nn_crops(nx, ny, nz, pin + pi * n, ptg + pi * n, p.batch, cx, cy, corners.data(), bin, btg, nn->stream);
    if (st != HZ_OK) return st;
    for (int b = 0; opl && b < 6; b += 2) {
      st = hz_nn_crops(nx, ny, nz, b6 + b * n, b6 + (b + 1) * n, p.batch, cx, cy, corners.data(), bcr + b * cn,
                       bcr + (b + 1) * cn, nn->stream);
      if (st != HZ_OK) return st;
    }
    double loss = 0.0;
    const NnGrid cg{cx, p.batch * cy, nz, cy, 0, (int64_t)cx * p.batch * cy * nz};
    // the residual needs one more column of exact network output around it
    st = opl ? nn_train_step(nn, cg, kHalo + 1, bin, btg, bcr, p.lr, p.clip, &loss)
             : nn_train_step(nn, cg, kHalo, bin, btg, nullptr, p.lr, p.clip, &loss);
    if (st != HZ_OK) return st;
    if (losses) losses[it] = loss;
  }
  NN_CK(cudaStreamSynchronize(nn->stream));
  return HZ_OK;
}

}  // extern "C"

