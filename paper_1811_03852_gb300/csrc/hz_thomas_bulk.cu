// hz_thomas_bulk.cu -- the per-column tridiagonal preconditioner (Maynard &
// Walters Sec. 2: C = T^-1 with the LU of T pre-computed at each horizontal
// point) with its fused vector update, staged through shared memory by bulk
// copies (sm_100+ cp.async.bulk, completion on mbarriers).
//
// A CTA owns a tile of kTC consecutive columns (column index j*nx + i) and
// marches the levels.  One producer warp copies, level by level, every input
// array's kTC-value row of the tile into a ring of kStages shared-memory
// slots; kTC consumer threads (one column each) wait for a slot, run the
// recurrence and release the slot.  Forward sweep: slot = one level's inputs
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

constexpr int kTC = 256;                        // columns per tile = consumer threads
constexpr int kConsumerWarps = kTC / 32;
constexpr int kBulkThreads = kTC + 32;          // + the producer warp
constexpr int kStages = 8;                      // ring slots
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
// ran out or another thread of the CTA gave up first
__device__ __forceinline__ bool mb_wait(unsigned bar, unsigned parity, const volatile int* abort) {
  if (mb_try(bar, parity)) return true;
  const unsigned long long t0 = gtimer();
  while (!mb_try(bar, parity)) {
    if (*abort) return false;
    if (gtimer() - t0 > (unsigned long long)kWaitNs) return false;
  }
  return true;
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

// bytes (a multiple of 16) from global src (16-byte aligned) to shared dst, completing on bar
__device__ __forceinline__ void bulk_copy(unsigned dst, const void* src, unsigned bytes, unsigned bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

}  // namespace

// MODE 0: q = r + beta (p - omega v) stored to p, z = T^-1 q to ph  (k_pre_p)
// MODE 1: q = r - alpha v stored to s, z = T^-1 q to sh               (k_pre_s)
// MODE 2: q = r (not stored), z = T^-1 r to out                       (T^-1 alone)
// err: device error word (bit 0: a bounded wait ran out).
template <int MODE>
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
            for (int q = 0; q < NIN; ++q) bulk_copy(dst + q * kRowBytes, src[q] + off, bytes, full0 + 8u * s);
          } else {  // back: the c' rows of levels k0, k0-1, ..., down to 0 at most kMaxIn of them
            const int k0 = nz - 1 - (step - nz) * kMaxIn;
            const int cnt = k0 + 1 < kMaxIn ? k0 + 1 : kMaxIn;
            mb_expect(full0 + 8u * s, (unsigned)cnt * bytes);
            for (int q = 0; q < cnt; ++q)
              bulk_copy(dst + q * kRowBytes, a.cp + (int64_t)(k0 - q) * ncol + c0, bytes, full0 + 8u * s);
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
    // ---- consumers: one column each --------------------------------------------
    const float beta = MODE == 0 ? (float)ctl->beta : 0.f;
    const float omega = MODE == 0 ? (float)ctl->omega : 0.f;
    const float alpha = MODE == 1 ? (float)ctl->alpha : 0.f;
    uint32_t use = 0;
    bool ok = true;
    for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
      const int64_t c0 = tile * kTC;
      const bool live = c0 + tid < ncol;
      float y = 0.f;
      for (int k = 0; k < nz; ++k, ++use) {
        const int s = (int)(use % kStages);
        // warp-uniform: the lanes meet at __syncwarp below
        if (!__all_sync(0xffffffffu, mb_wait(full0 + 8u * s, (use / kStages) & 1u, abort))) {
          ok = false;
          break;
        }
        const float* sl = ring + (size_t)s * (kSlotBytes / 4);
        if (live) {
          float q, m, l;
          if (MODE == 0) {
            q = fmaf(beta, fmaf(-omega, sl[2 * kTC + tid], sl[kTC + tid]), sl[tid]);
            m = sl[3 * kTC + tid];
            l = sl[4 * kTC + tid];
          } else if (MODE == 1) {
            q = fmaf(-alpha, sl[kTC + tid], sl[tid]);
            m = sl[2 * kTC + tid];
            l = sl[3 * kTC + tid];
          } else {
            q = sl[tid];
            m = sl[kTC + tid];
            l = sl[2 * kTC + tid];
          }
          const int64_t idx = (int64_t)k * ncol + c0 + tid;
          if (MODE != 2) stw<float, ST_EF>(qout + idx, q);
          y = fmaf(m, q, -l * y);
          stw<float, ST_EL>(zout + idx, y);  // parked until the back sweep
        }
        __syncwarp();
        if (lane == 0) mb_arrive(empty0 + 8u * s);
      }
      if (!ok) break;
      float zn = 0.f;
      for (int k0 = nz - 1; k0 >= 0; k0 -= kMaxIn, ++use) {
        const int s = (int)(use % kStages);
        if (!__all_sync(0xffffffffu, mb_wait(full0 + 8u * s, (use / kStages) & 1u, abort))) {
          ok = false;
          break;
        }
        if (live) {
          const float* sl = ring + (size_t)s * (kSlotBytes / 4);
          const int cnt = k0 + 1 < kMaxIn ? k0 + 1 : kMaxIn;
          float yk[kMaxIn];
#pragma unroll
          for (int q = 0; q < kMaxIn; ++q)  // the group's parked values, all loads first
            if (q < cnt) yk[q] = zout[(int64_t)(k0 - q) * ncol + c0 + tid];
#pragma unroll
          for (int q = 0; q < kMaxIn; ++q) {
            if (q < cnt) {
              zn = fmaf(-sl[q * kTC + tid], zn, yk[q]);
              stw<float, ST_EF>(zout + (int64_t)(k0 - q) * ncol + c0 + tid, zn);
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

size_t thomas_bulk_smem(int) { return (size_t)kStages * kSlotBytes + 2 * kStages * 8 + 16; }

bool thomas_bulk_ok(const Grid& g) { return g.ncol % 4 == 0; }

template <int MODE>
static cudaError_t bulk_prepare() {
  static bool done = false;  // the attribute is per function
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_thomas_bulk<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)thomas_bulk_smem(0));
  if (e == cudaSuccess) done = true;
  return e;
}

int thomas_bulk_grid(const Grid& g, const Launch& L, int mode) {
  const void* k = mode == 0 ? (const void*)k_thomas_bulk<0> : mode == 1 ? (const void*)k_thomas_bulk<1>
                                                                          : (const void*)k_thomas_bulk<2>;
  const int64_t tiles = (g.ncol + kTC - 1) / kTC;
  return grid_for(k, kBulkThreads, L, tiles, thomas_bulk_smem(g.nz));
}

cudaError_t launch_thomas_bulk(int mode, const Grid& g, const Bands<float>& a, const Vecs<float>& w, const float* r,
                               float* z, Ctl* ctl, int* err, const Launch& L) {
  if (!thomas_bulk_ok(g)) return cudaErrorInvalidValue;
  const size_t sm = thomas_bulk_smem(g.nz);
  cudaError_t e = mode == 0 ? bulk_prepare<0>() : mode == 1 ? bulk_prepare<1>() : bulk_prepare<2>();
  if (e != cudaSuccess) return e;
  const int grid = thomas_bulk_grid(g, L, mode);
  if (mode == 0)
    k_thomas_bulk<0><<<grid, kBulkThreads, sm, L.stream>>>(g, a, w, nullptr, nullptr, ctl, err);
  else if (mode == 1)
    k_thomas_bulk<1><<<grid, kBulkThreads, sm, L.stream>>>(g, a, w, nullptr, nullptr, ctl, err);
  else
    k_thomas_bulk<2><<<grid, kBulkThreads, sm, L.stream>>>(g, a, w, r, z, ctl, err);
  return cudaGetLastError();
}

// occupancy queries outside any stream capture (the attribute first)
void warm_thomas_bulk(const Launch& L, int nz) {
  Grid g{1, 1, nz, 4, 4 * (int64_t)nz};
  if (bulk_prepare<0>() != cudaSuccess || bulk_prepare<1>() != cudaSuccess || bulk_prepare<2>() != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  for (int m = 0; m < 3; ++m) thomas_bulk_grid(g, L, m);
}

}  // namespace hz
