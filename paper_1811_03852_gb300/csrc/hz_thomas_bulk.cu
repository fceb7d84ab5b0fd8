// hz_thomas_bulk.cu -- the per-column tridiagonal preconditioner (Maynard &
// Walters Sec. 2: C = T^-1 with the LU of T pre-computed at each horizontal
// point) with its fused vector update, staged through shared memory by bulk
// copies (sm_100+ cp.async.bulk, completion on mbarriers).
//
// A CTA owns a tile of kTC consecutive columns (column index j*nx + i) and
// marches the levels.  One producer warp copies, level by level, every input
// array's kTC-value row of the tile (4 KB) into a ring of kStages
// shared-memory slots; kTC / 4 consumer threads (four adjacent columns each,
// float4 reads of the slot) wait for a slot, run the recurrences and release
// the slot.  Forward sweep: slot = one level's inputs
// (r, and p, v or v for the axpy; the factors m, l); the consumer forms q
// (p = r + beta (p - omega v), s = r - alpha v, or q = r), stores it, and
// parks y_k = m_k q_k - l_k y_(k-1) in the output vector with the L2
// evict-last priority.  Back sweep: slot = the c' rows of up to kMaxIn levels
// (descending); the consumer reads back those levels' y (its own stores, an
// L2 hit) and stores z_k = y_k - c'_k z_(k+1) over them, evict-first.  The
// small ring (kStages slots) leaves room for several CTAs, hence several
// producers, per SM; the memory parallelism comes from the copies in flight,
// not from registers.  DRAM traffic per point: the inputs and c' once, q and
// z once -- the algorithmic bytes.
//
// Every wait is bounded by %globaltimer: a wait that runs out sets the error
// word, the CTA stops issuing, waits (bounded) for the copies it issued, and
// returns; the host reports HZ_ERR_TIMEOUT.
#include "hz_krylov.cuh"

namespace hz {

namespace {

constexpr int kTC = 1024;                       // columns per tile
constexpr int kCV = 4;                          // columns per consumer thread
constexpr int kConsumers = kTC / kCV;
constexpr int kConsumerWarps = kConsumers / 32;
constexpr int kBulkThreads = kConsumers + 32;   // + the producer warp
// ring slots: a template parameter of the kernel (3, 4 or 5; the variant table's depth)
constexpr int kMaxIn = 5;                       // input rows per slot at most
constexpr unsigned kRowBytes = kTC * 4;         // one array's row of a tile
constexpr unsigned kSlotBytes = kMaxIn * kRowBytes;
constexpr long long kWaitNs = 1000000000LL;     // bound of every wait (1 s)

__device__ __forceinline__ unsigned su32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool mb_try(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// wait for the completion of the phase with this parity; false if the bound
// ran out or another thread of the CTA gave up first (the timer and the abort
// flag are read every 32 polls: each try_wait already suspends the thread for
// a while)
__device__ __forceinline__ bool mb_wait(unsigned bar, unsigned parity, const volatile int* abort) {
  if (mb_try(bar, parity)) return true;
  const unsigned long long t0 = gtimer();
  for (unsigned it = 1;; ++it) {
    if (mb_try(bar, parity)) return true;
    if ((it & 31u) == 0) {
      if (*abort) return false;
      if (gtimer() - t0 > (unsigned long long)kWaitNs) return false;
    }
  }
}

// the same without the abort test: the drain of copies still in flight
__device__ __forceinline__ bool mb_wait_drain(unsigned bar, unsigned parity) {
  if (mb_try(bar, parity)) return true;
  const unsigned long long t0 = gtimer();
  while (!mb_try(bar, parity))
    if (gtimer() - t0 > (unsigned long long)kWaitNs) return false;
  return true;
}

__device__ __forceinline__ void mb_arrive(unsigned bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mb_expect(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// bytes (a multiple of 16) from global src (16-byte aligned) to shared dst,
// completing on bar; pol: the L2 policy of the source lines (the copies
// stream arrays read once per launch, evict-first, so that the parked
// forward sweep keeps its place in L2 for the back sweep)
__device__ __forceinline__ void bulk_copy(unsigned dst, const void* src, unsigned bytes, unsigned bar, uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(bar), "l"(pol)
      : "memory");
}

}  // namespace

// MODE 0: q = r + beta (p - omega v) stored to p, z = T^-1 q to ph  (k_pre_p)
// MODE 1: q = r - alpha v stored to s, z = T^-1 q to sh               (k_pre_s)
// MODE 2: q = r (not stored), z = T^-1 r to out                       (T^-1 alone)
// err: device error word (bit 0: a bounded wait ran out).
template <int MODE, int kStages>
__global__ void __launch_bounds__(kBulkThreads) k_thomas_bulk(Grid g, Bands<float> a, Vecs<float> w, const float* r_in,
                                                              float* z_out, Ctl* ctl, int* err) {
  constexpr int NIN = MODE == 0 ? 5 : MODE == 1 ? 4 : 3;  // rows per forward slot
  if (MODE == 0 && (ctl->state != ST_RUNNING || ctl->fresh)) return;
  if (MODE == 1 && ctl->state != ST_RUNNING) return;
  extern __shared__ __align__(128) unsigned char smem[];
  float* ring = reinterpret_cast<float*>(smem);                                 // [kStages][kMaxIn][kTC]
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kStages * kSlotBytes);
  volatile int* abort = reinterpret_cast<volatile int*>(bars + 2 * kStages);
  const unsigned full0 = su32(bars), empty0 = su32(bars + kStages);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(full0 + 8u * s) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(empty0 + 8u * s), "r"(kConsumerWarps) : "memory");
    }
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  const int64_t ncol = g.ncol;
  const int nz = g.nz;
  const int64_t ntiles = (ncol + kTC - 1) / kTC;
  const int nback = (nz + kMaxIn - 1) / kMaxIn;  // back-sweep slots per tile (kMaxIn levels each)
  const int nuse = nz + nback;                   // slot uses per tile
  // the inputs of the forward sweep, in slot-row order
  const float* rin = r_in;
  float* qout = nullptr;
  float* zout = z_out;
  if (MODE == 0) {
    rin = ctl->rsel ? w.r : w.rhs;
    qout = w.p;
    zout = w.ph;
  } else if (MODE == 1) {
    rin = ctl->rsel ? w.r : w.rhs;
    qout = w.s;
    zout = w.sh;
  }
  const float* src[kMaxIn];
  if (MODE == 0) {
    src[0] = rin; src[1] = w.p; src[2] = w.v; src[3] = a.m; src[4] = a.l;
  } else if (MODE == 1) {
    src[0] = rin; src[1] = w.v; src[2] = a.m; src[3] = a.l; src[4] = nullptr;
  } else {
    src[0] = rin; src[1] = a.m; src[2] = a.l; src[3] = nullptr; src[4] = nullptr;
  }

  if (warp == kConsumerWarps) {
    // ---- producer: one lane issues every copy ----------------------------------
    if (lane == 0) {
      uint32_t use = 0;  // slot uses issued (slot = use % kStages, its phase = use / kStages)
      bool ok = true;
      const uint64_t pol = l2_evict_first();
      for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int64_t c0 = tile * kTC;
        const unsigned bytes = (unsigned)((ncol - c0 < kTC ? ncol - c0 : kTC) * 4);
        for (int step = 0; step < nuse && ok; ++step, ++use) {
          const int s = (int)(use % kStages);
          const uint32_t u = use / kStages;
          if (u > 0 && !mb_wait(empty0 + 8u * s, (u - 1) & 1u, abort)) {
            ok = false;
            break;
          }
          const unsigned dst = su32(ring) + (unsigned)s * kSlotBytes;
          if (step < nz) {  // forward: level k's inputs
            const int64_t off = (int64_t)step * ncol + c0;
            mb_expect(full0 + 8u * s, NIN * bytes);
#pragma unroll
            for (int q = 0; q < NIN; ++q) bulk_copy(dst + q * kRowBytes, src[q] + off, bytes, full0 + 8u * s, pol);
          } else {  // back: the c' rows of levels k0, k0-1, ..., down to 0 at most kMaxIn of them
            const int k0 = nz - 1 - (step - nz) * kMaxIn;
            const int cnt = k0 + 1 < kMaxIn ? k0 + 1 : kMaxIn;
            mb_expect(full0 + 8u * s, (unsigned)cnt * bytes);
            for (int q = 0; q < cnt; ++q)
              bulk_copy(dst + q * kRowBytes, a.cp + (int64_t)(k0 - q) * ncol + c0, bytes, full0 + 8u * s, pol);
          }
        }
      }
      if (!ok) {
        atomicOr(err, 1);
        *abort = 1;
      }
      // the copies still in flight land before the CTA's shared memory is released
      const uint32_t first = use > kStages ? use - kStages : 0;
      for (uint32_t v = first; v < use; ++v) mb_wait_drain(full0 + 8u * (v % kStages), (v / kStages) & 1u);
    }
  } else {
    // ---- consumers: kCV adjacent columns each ------------------------------------
    const float beta = MODE == 0 ? (float)ctl->beta : 0.f;
    const float omega = MODE == 0 ? (float)ctl->omega : 0.f;
    const float alpha = MODE == 1 ? (float)ctl->alpha : 0.f;
    const int c = tid * kCV;  // first column of this thread within the tile
    uint32_t use = 0;
    bool ok = true;
    for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
      const int64_t c0 = tile * kTC;
      const bool live = c0 + c < ncol;  // the tile width is a multiple of 4: all kCV columns or none
      float y[kCV] = {0.f, 0.f, 0.f, 0.f};
      for (int k = 0; k < nz; ++k, ++use) {
        const int s = (int)(use % kStages);
        // warp-uniform: the lanes meet at __syncwarp below
        if (!__all_sync(0xffffffffu, mb_wait(full0 + 8u * s, (use / kStages) & 1u, abort))) {
          ok = false;
          break;
        }
        const float* sl = ring + (size_t)s * (kSlotBytes / 4);
        if (live) {
          const float4 r4 = *reinterpret_cast<const float4*>(sl + c);
          float4 q4, m4, l4;
          if (MODE == 0) {
            const float4 p4 = *reinterpret_cast<const float4*>(sl + kTC + c);
            const float4 v4 = *reinterpret_cast<const float4*>(sl + 2 * kTC + c);
            m4 = *reinterpret_cast<const float4*>(sl + 3 * kTC + c);
            l4 = *reinterpret_cast<const float4*>(sl + 4 * kTC + c);
            q4.x = fmaf(beta, fmaf(-omega, v4.x, p4.x), r4.x);
            q4.y = fmaf(beta, fmaf(-omega, v4.y, p4.y), r4.y);
            q4.z = fmaf(beta, fmaf(-omega, v4.z, p4.z), r4.z);
            q4.w = fmaf(beta, fmaf(-omega, v4.w, p4.w), r4.w);
          } else if (MODE == 1) {
            const float4 v4 = *reinterpret_cast<const float4*>(sl + kTC + c);
            m4 = *reinterpret_cast<const float4*>(sl + 2 * kTC + c);
            l4 = *reinterpret_cast<const float4*>(sl + 3 * kTC + c);
            q4.x = fmaf(-alpha, v4.x, r4.x);
            q4.y = fmaf(-alpha, v4.y, r4.y);
            q4.z = fmaf(-alpha, v4.z, r4.z);
            q4.w = fmaf(-alpha, v4.w, r4.w);
          } else {
            q4 = r4;
            m4 = *reinterpret_cast<const float4*>(sl + kTC + c);
            l4 = *reinterpret_cast<const float4*>(sl + 2 * kTC + c);
          }
          const int64_t idx = (int64_t)k * ncol + c0 + c;
          if (MODE != 2) stw<float4, ST_EF>(reinterpret_cast<float4*>(qout + idx), q4);
          y[0] = fmaf(m4.x, q4.x, -l4.x * y[0]);
          y[1] = fmaf(m4.y, q4.y, -l4.y * y[1]);
          y[2] = fmaf(m4.z, q4.z, -l4.z * y[2]);
          y[3] = fmaf(m4.w, q4.w, -l4.w * y[3]);
          // parked until the back sweep
          stw<float4, ST_EL>(reinterpret_cast<float4*>(zout + idx), make_float4(y[0], y[1], y[2], y[3]));
        }
        __syncwarp();
        if (lane == 0) mb_arrive(empty0 + 8u * s);
      }
      if (!ok) break;
      float zn[kCV] = {0.f, 0.f, 0.f, 0.f};
      for (int k0 = nz - 1; k0 >= 0; k0 -= kMaxIn, ++use) {
        const int s = (int)(use % kStages);
        if (!__all_sync(0xffffffffu, mb_wait(full0 + 8u * s, (use / kStages) & 1u, abort))) {
          ok = false;
          break;
        }
        if (live) {
          const float* sl = ring + (size_t)s * (kSlotBytes / 4);
          const int cnt = k0 + 1 < kMaxIn ? k0 + 1 : kMaxIn;
          float4 yk[kMaxIn];
#pragma unroll
          for (int q = 0; q < kMaxIn; ++q)  // the group's parked values, all loads first
            if (q < cnt) yk[q] = *reinterpret_cast<const float4*>(zout + (int64_t)(k0 - q) * ncol + c0 + c);
#pragma unroll
          for (int q = 0; q < kMaxIn; ++q) {
            if (q < cnt) {
              const float4 c4 = *reinterpret_cast<const float4*>(sl + q * kTC + c);
              zn[0] = fmaf(-c4.x, zn[0], yk[q].x);
              zn[1] = fmaf(-c4.y, zn[1], yk[q].y);
              zn[2] = fmaf(-c4.z, zn[2], yk[q].z);
              zn[3] = fmaf(-c4.w, zn[3], yk[q].w);
              stw<float4, ST_EF>(reinterpret_cast<float4*>(zout + (int64_t)(k0 - q) * ncol + c0 + c),
                                 make_float4(zn[0], zn[1], zn[2], zn[3]));
            }
          }
        }
        __syncwarp();
        if (lane == 0) mb_arrive(empty0 + 8u * s);
      }
    }
    if (!ok && lane == 0) {
      atomicOr(err, 1);
      *abort = 1;
    }
  }
  __syncthreads();
}

size_t thomas_bulk_smem(int stages) { return (size_t)stages * kSlotBytes + 2 * stages * 8 + 16; }

bool thomas_bulk_ok(const Grid& g) { return g.ncol % 4 == 0; }

template <int MODE, int S>
static cudaError_t bulk_prepare() {
  static bool done = false;  // the attribute is per function
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_thomas_bulk<MODE, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)thomas_bulk_smem(S));
  if (e == cudaSuccess) done = true;
  return e;
}

template <int S>
static cudaError_t launch_s(int mode, int cap, const Grid& g, const Bands<float>& a, const Vecs<float>& w,
                            const float* r, float* z, Ctl* ctl, int* err, const Launch& L) {
  const size_t sm = thomas_bulk_smem(S);
  const int64_t tiles = (g.ncol + kTC - 1) / kTC;
  cudaError_t e;
  if (mode == 0) {
    if ((e = bulk_prepare<0, S>()) != cudaSuccess) return e;
    const int grid = grid_for((const void*)k_thomas_bulk<0, S>, kBulkThreads, L, tiles, sm, cap);
    k_thomas_bulk<0, S><<<grid, kBulkThreads, sm, L.stream>>>(g, a, w, nullptr, nullptr, ctl, err);
  } else if (mode == 1) {
    if ((e = bulk_prepare<1, S>()) != cudaSuccess) return e;
    const int grid = grid_for((const void*)k_thomas_bulk<1, S>, kBulkThreads, L, tiles, sm, cap);
    k_thomas_bulk<1, S><<<grid, kBulkThreads, sm, L.stream>>>(g, a, w, nullptr, nullptr, ctl, err);
  } else {
    if ((e = bulk_prepare<2, S>()) != cudaSuccess) return e;
    const int grid = grid_for((const void*)k_thomas_bulk<2, S>, kBulkThreads, L, tiles, sm, cap);
    k_thomas_bulk<2, S><<<grid, kBulkThreads, sm, L.stream>>>(g, a, w, r, z, ctl, err);
  }
  return cudaGetLastError();
}

cudaError_t launch_thomas_bulk(int mode, int stages, int per_sm_cap, const Grid& g, const Bands<float>& a,
                               const Vecs<float>& w, const float* r, float* z, Ctl* ctl, int* err, const Launch& L) {
  if (!thomas_bulk_ok(g)) return cudaErrorInvalidValue;
  if (stages == 3) return launch_s<3>(mode, per_sm_cap, g, a, w, r, z, ctl, err, L);
  if (stages == 4) return launch_s<4>(mode, per_sm_cap, g, a, w, r, z, ctl, err, L);
  if (stages == 5) return launch_s<5>(mode, per_sm_cap, g, a, w, r, z, ctl, err, L);
  if (stages == 8) return launch_s<8>(mode, per_sm_cap, g, a, w, r, z, ctl, err, L);
  return cudaErrorInvalidValue;
}

// attributes and occupancy queries outside any stream capture
template <int S>
static void warm_s(const Launch& L) {
  if (bulk_prepare<0, S>() != cudaSuccess || bulk_prepare<1, S>() != cudaSuccess ||
      bulk_prepare<2, S>() != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  const size_t sm = thomas_bulk_smem(S);
  grid_for((const void*)k_thomas_bulk<0, S>, kBulkThreads, L, 1, sm);
  grid_for((const void*)k_thomas_bulk<1, S>, kBulkThreads, L, 1, sm);
  grid_for((const void*)k_thomas_bulk<2, S>, kBulkThreads, L, 1, sm);
}
void warm_thomas_bulk(const Launch& L, int) {
  warm_s<3>(L);
  warm_s<4>(L);
  warm_s<5>(L);
  warm_s<8>(L);
}

}  // namespace hz
