// hz_nn_tc.cu -- the learned stage's 16 -> 16 and 16 -> 1 convolutions on the
// fifth-generation tensor cores: tcgen05.mma from shared-memory descriptors,
// FP32 accumulators in tensor memory (TMEM), BF16 operands.
//
// A CTA owns a tile of kTI = 128 consecutive points in each of kTJ = 2 rows
// and marches k.  Input levels k-1, k, k+1 sit in a ring of shared-memory
// planes (130 x 4 points with the halo, the two 8-channel halves of a point in
// separate half-planes) filled by cp.async two levels ahead.  For each row and
// tap one thread issues an M = 128, N = 16, K = 16 MMA whose A operand is the
// row's 128 points shifted by the tap (a K-major, unswizzled operand: core
// matrices of 8 points x 8 channels are 128 contiguous bytes, 128 B apart
// along M, one half-plane apart along K) and whose B operand is the tap's
// 16 x 16 weight block.  Level k accumulates in one of two TMEM buffers while
// the four warps read level k-1 out of the other (tcgen05.ld, one point and
// its 16 channels per thread), add the bias, apply GELU and store.
//
// Every wait is bounded: a tensor-core completion that does not arrive within
// the limit sets *err, the level's epilogue is skipped (its output is then
// invalid), and the CTA stops: it waits (bounded) for the commits still
// outstanding, frees its TMEM and returns.
#include "hz_nn.cuh"

namespace hz {

namespace {

constexpr int kTI = 128, kTJ = 2;
constexpr int kPI = kTI + 2, kPJ = kTJ + 2, kPP = kPI * kPJ;  // plane with halo: 130 x 4 points
constexpr int kRing = 6;                // plane slots: levels k-2 .. k+kAhead in flight or in use
constexpr int kAhead = kRing - 3;        // copies of level k + kAhead start at level k
constexpr unsigned kHalfBytes = kPP * 16;        // one 8-channel half of a plane
constexpr unsigned kSlotBytes = 2 * kHalfBytes;  // one ring slot
constexpr unsigned kWBytes = kTaps * 512;        // B operands: [tap][channel half][co][8 ci] BF16
constexpr unsigned kUsedBytes = kRing * kSlotBytes + kWBytes + 256;
// dynamic shared memory per CTA (97 KB: two CTAs per SM)
constexpr unsigned kSmemBytes = kUsedBytes;
constexpr int kCtasPerSm = kUsedBytes * 2 + 2048 <= 228 * 1024 ? 2 : 1;
static_assert(kUsedBytes <= kSmemBytes, "shared-memory layout");
constexpr int kTmemCols = 64;                    // two buffers x two rows x 16 columns
constexpr long long kWaitLimitNs = 500000000LL;  // bound of a completion wait
// instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major, N = 16, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);

struct Geo {
  int i0, j0;
  bool jlo_zero, jhi_zero;
};

__device__ __forceinline__ Geo tc_geo(const NnGrid& g, int64_t tile, int tiles_i) {
  Geo t;
  t.i0 = (int)(tile % tiles_i) * kTI;
  t.j0 = (int)(tile / tiles_i) * kTJ;
  t.jlo_zero = (t.j0 % g.seg) == 0;
  t.jhi_zero = ((t.j0 + kTJ) % g.seg) == 0;
  return t;
}

// source point (level 0) of plane position (ti, tj), or -1 for a zero
__device__ __forceinline__ int64_t tc_src(const NnGrid& g, const Geo& t, int ti, int tj) {
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
  return (int64_t)gj * g.nx + gi;
}

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// shared-memory matrix descriptor: start, leading (K-direction) and stride
// (M/N-direction) byte offsets of the core matrices, descriptor version 1,
// no swizzle
__device__ __forceinline__ uint64_t umma_desc(unsigned saddr, unsigned lbo, unsigned sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

__device__ __forceinline__ void umma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(unsigned mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ bool mbar_try(unsigned mbar, unsigned parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(mbar), "r"(parity)
      : "memory");
  return done != 0;
}

__device__ __forceinline__ bool mbar_wait(unsigned mbar, unsigned parity) {
  if (mbar_try(mbar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  while (!mbar_try(mbar, parity))
    if (globaltimer() - t0 > (unsigned long long)kWaitLimitNs) return false;
  return true;
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld1(uint32_t taddr, uint32_t& v) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(v) : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// per-thread copy list of a tile's plane (chunks q = thread + 128 m of 2 * kPP)
struct TcCopy {
  static constexpr int kMax = (2 * kPP + 127) / 128;
  int64_t src[kMax];  // element offset within a level (-1: zero fill, -2: none)
  unsigned dst[kMax];
  __device__ __forceinline__ void init(const NnGrid& g, const Geo& t) {
#pragma unroll
    for (int m = 0; m < kMax; ++m) {
      const int q = threadIdx.x + 128 * m;
      src[m] = -2;
      if (q < 2 * kPP) {
        const int pp = q >> 1, hh = q & 1;
        const int64_t s = tc_src(g, t, pp % kPI, pp / kPI);
        src[m] = s >= 0 ? s * kC + hh * 8 : -1;
        dst[m] = hh * kHalfBytes + pp * 16;
      }
    }
  }
  __device__ __forceinline__ void issue(unsigned slot, const __nv_bfloat16* h, int64_t kofs) const {
#pragma unroll
    for (int m = 0; m < kMax; ++m) {
      if (src[m] == -2) continue;
      const bool ok = src[m] >= 0;
      const void* gp = ok ? (const void*)(h + kofs + src[m]) : (const void*)h;
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(slot + dst[m]), "l"(gp), "r"(ok ? 16 : 0)
                   : "memory");
    }
  }
};

}  // namespace

// MODE 0: 16 -> 16 + bias, z (optional), hout = bf16(gelu).  MODE 1: 16 -> 1 + bias -> out (or base + sigma y).
template <int MODE>
__global__ void __launch_bounds__(128, kCtasPerSm) k_nn_tc(NnGrid g, const __nv_bfloat16* __restrict__ hin,
                                                  const __nv_bfloat16* __restrict__ wb, const float* __restrict__ w4,
                                                  const float* __restrict__ bias, float* __restrict__ z,
                                                  __nv_bfloat16* __restrict__ hout, const float* base,
                                                  const double* nrm2, float* out, int* err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __nv_bfloat16* Wsm = reinterpret_cast<__nv_bfloat16*>(smem + kRing * kSlotBytes);
  float* Bs = reinterpret_cast<float*>(smem + kRing * kSlotBytes + kWBytes);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + kRing * kSlotBytes + kWBytes + 64);  // one per TMEM buffer
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + kRing * kSlotBytes + kWBytes + 128);
  int* abort_flag = reinterpret_cast<int*>(smem + kRing * kSlotBytes + kWBytes + 192);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // B operands: Wsm[t][kh][co][j] = W[t][co][8 kh + j]
  for (int q = tid; q < kTaps * 256; q += 128) {
    const int t = q >> 8, r = q & 255, kh = r >> 7, co = (r >> 3) & 15, j = r & 7;
    __nv_bfloat16 v;
    if (MODE == 0)
      v = wb[t * 256 + co * 16 + kh * 8 + j];
    else
      v = co == 0 ? __float2bfloat16_rn(w4[t * 16 + kh * 8 + j]) : __float2bfloat16_rn(0.f);
    Wsm[q] = v;
  }
  if (tid < kC) Bs[tid] = MODE == 0 ? bias[tid] : (tid == 0 ? bias[0] : 0.f);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar + 1)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");  // visible to the tensor core's arrive
    *abort_flag = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_async_smem();  // the weights, written by the generic proxy, are read by the tensor core
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const unsigned mb = smem_u32(mbar);
  const unsigned sbase = smem_u32(smem);
  const unsigned wbase = smem_u32(Wsm);
  // descriptors: A = row window in a slot (start field advanced per slot, row and tap), B = tap block
  const uint64_t adesc0 = umma_desc(sbase, kHalfBytes, 128);
  const uint64_t bdesc0 = umma_desc(wbase, 256, 128);

  float sigma = 1.f;
  if (MODE == 1 && nrm2) sigma = (float)sqrt(*nrm2 / (double)g.n);
  const int tiles_i = (g.nx + kTI - 1) / kTI;
  const int64_t ntiles = (int64_t)tiles_i * ((g.ny + kTJ - 1) / kTJ);
  const int64_t plane = (int64_t)g.nx * g.ny;
  unsigned phase = 0;        // bit b: parity of the next completion of barrier b
  unsigned outstanding = 0;  // bit b: a commit on barrier b whose completion has not been seen
  bool aborted = false;
  for (int64_t tile = blockIdx.x; tile < ntiles && !aborted; tile += gridDim.x) {
    const Geo t = tc_geo(g, tile, tiles_i);
    TcCopy pc;
    pc.init(g, t);
    __syncthreads();  // the previous tile's MMAs and readers are done with the ring
    for (int kq = 0; kq < kAhead; ++kq) {
      if (kq < g.nz) pc.issue(sbase + kq * kSlotBytes, hin, (int64_t)kq * plane * kC);
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
    asm volatile("cp.async.wait_group %0;" ::"n"(kAhead - 2) : "memory");  // levels 0 and 1 landed
    fence_async_smem();
    __syncthreads();
    // level k: copies of k+3 start, the MMAs of k are queued behind those of
    // k-1, then the epilogue of k-1 waits for its MMAs and reads its buffer
    for (int k = 0; k <= g.nz; ++k) {
      if (k + kAhead < g.nz)
        pc.issue(sbase + ((k + kAhead) % kRing) * kSlotBytes, hin, (int64_t)(k + kAhead) * plane * kC);
      asm volatile("cp.async.commit_group;" ::: "memory");
      if (k < g.nz && tid == 0) {
        tc_fence_after();
        const bool has[3] = {k > 0, true, k + 1 < g.nz};
        const unsigned sl[3] = {((k + kRing - 1) % kRing) * kSlotBytes, (k % kRing) * kSlotBytes,
                                ((k + 1) % kRing) * kSlotBytes};
        uint32_t acc = 0;  // the rows' accumulator chains are interleaved tap by tap
#pragma unroll
        for (int tp = 0; tp < kTaps; ++tp) {
          const int dk = tp / 9, dj = (tp / 3) % 3 - 1, di = tp % 3 - 1;
          if (!has[dk]) continue;
#pragma unroll
          for (int r = 0; r < kTJ; ++r) {
            const uint32_t dcol = tmem + (uint32_t)((k & 1) * (kTJ * 16) + r * 16);
            const unsigned off = sl[dk] + (unsigned)(((r + 1 + dj) * kPI + 1 + di) * 16);
            umma(dcol, adesc0 + (off >> 4), bdesc0 + (uint64_t)(tp * 32), acc);
          }
          acc = 1;
        }
        umma_commit(mb + 8u * (k & 1));
      }
      if (k < g.nz) outstanding |= 1u << (k & 1);
      bool level_ok = true;
      if (k >= 1) {  // the MMAs of level k-1 are complete: its TMEM buffer is readable
        const unsigned b = (k - 1) & 1;
        // warp-uniform decision: tcgen05.ld below is .sync.aligned, so a warp
        // reads the buffer only if every lane saw the completion
        level_ok = __all_sync(0xffffffffu, mbar_wait(mb + 8u * b, (phase >> b) & 1u));
        if (level_ok) {
          phase ^= 1u << b;
          outstanding &= ~(1u << b);
        } else if (lane == 0) {
          atomicExch(abort_flag, 1);
          atomicExch(err, 1);
        }
        tc_fence_after();
      }
      if (k >= 1 && level_ok) {  // epilogue of level k-1 (skipped, output invalid, once a wait gave up)
        const int kk = k - 1;
        const int gi = t.i0 + 32 * warp + lane;
#pragma unroll
        for (int r = 0; r < kTJ; ++r) {
          const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)((kk & 1) * (kTJ * 16) + r * 16);
          const int gj = t.j0 + r;
          const bool valid = gi < g.nx && gj < g.ny;
          const int64_t p = (int64_t)kk * plane + (int64_t)gj * g.nx + gi;
          if (MODE == 0) {
            uint32_t v[16];
            tmem_ld16(taddr, v);
            tmem_wait_ld();
            if (valid) {
              float a[kC];
#pragma unroll
              for (int c = 0; c < kC; ++c) a[c] = __uint_as_float(v[c]) + Bs[c];
              if (z) {
#pragma unroll
                for (int c = 0; c < kC; c += 4)
                  *reinterpret_cast<float4*>(z + p * kC + c) = make_float4(a[c], a[c + 1], a[c + 2], a[c + 3]);
              }
              __align__(16) __nv_bfloat16 hv[kC];
#pragma unroll
              for (int c = 0; c < kC; ++c) hv[c] = __float2bfloat16_rn(gelu_f(a[c]));
              reinterpret_cast<uint4*>(hout + p * kC)[0] = reinterpret_cast<const uint4*>(hv)[0];
              reinterpret_cast<uint4*>(hout + p * kC)[1] = reinterpret_cast<const uint4*>(hv)[1];
            }
          } else {
            uint32_t v;
            tmem_ld1(taddr, v);
            tmem_wait_ld();
            if (valid) {
              const float y = __uint_as_float(v) + Bs[0];
              out[p] = base ? fmaf(sigma, y, base[p]) : y;
            }
          }
        }
        tc_fence_before();
      }
      asm volatile("cp.async.wait_group %0;" ::"n"(kAhead - 2) : "memory");  // level k+2 landed
      fence_async_smem();
      __syncthreads();
      if (*abort_flag) {
        aborted = true;
        break;
      }
    }
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  // after an abort, MMAs committed to a barrier whose completion was not seen
  // may still be writing TMEM: wait for them (again bounded) before freeing it.
  // If such a wait also gives up, the CTA frees its TMEM regardless (a CTA
  // must not exit holding it); *err is already set and the output is invalid.
  for (unsigned b = 0; b < 2; ++b)
    if (outstanding & (1u << b)) mbar_wait(mb + 8u * b, (phase >> b) & 1u);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

bool nn_tc_ok(const NnGrid& g) { return g.nx >= kTI && (g.seg == g.ny || g.seg % kTJ == 0); }

static int tc_grid(const NnGrid& g, int sms) {
  const int64_t tiles = (int64_t)((g.nx + kTI - 1) / kTI) * ((g.ny + kTJ - 1) / kTJ);
  return (int)std::min<int64_t>(tiles, (int64_t)sms * kCtasPerSm);
}

template <int MODE>
static cudaError_t tc_prepare() {
  static bool done = false;  // attribute set once per process (same value on every device)
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_nn_tc<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
  if (e == cudaSuccess) done = true;
  return e;
}

cudaError_t nn_tc_mid(const NnGrid& g, const __nv_bfloat16* hin, const __nv_bfloat16* wb, const float* bias, float* z,
                      __nv_bfloat16* hout, int* err, int sms, cudaStream_t s) {
  cudaError_t e = tc_prepare<0>();
  if (e != cudaSuccess) return e;
  k_nn_tc<0><<<tc_grid(g, sms), 128, kSmemBytes, s>>>(g, hin, wb, nullptr, bias, z, hout, nullptr, nullptr, nullptr,
                                                      err);
  return cudaGetLastError();
}

cudaError_t nn_tc_l4(const NnGrid& g, const __nv_bfloat16* hin, const float* w4, const float* b4, const float* base,
                     const double* nrm2, float* out, int* err, int sms, cudaStream_t s) {
  cudaError_t e = tc_prepare<1>();
  if (e != cudaSuccess) return e;
  k_nn_tc<1><<<tc_grid(g, sms), 128, kSmemBytes, s>>>(g, hin, nullptr, w4, b4, nullptr, nullptr, base, nrm2, out,
                                                      err);
  return cudaGetLastError();
}

}  // namespace hz
