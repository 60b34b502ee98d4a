// Batched D2Q9 sweep through shared memory: bands of whole rows moved by bulk
// asynchronous copies (the TMA engine's 1D form), collided in place in shared
// memory, and written back by bulk copies.
//
// A band is `rows` consecutive whole rows y0 .. y0 + rows - 1 of one run.  In
// the AA layout of either parity the band's slots for population j are whole
// rows of plane j: rows y0 + e_y .. y0 + e_y + rows - 1 (e_y of velocity j in
// the odd sweep, 0 in the even sweep).  Every element of those rows belongs to
// a node of the band, and to no other band.  So each (band, population) is one
// contiguous span of the population buffer:
//   * load:  one bulk copy of the span rounded out to 16-byte boundaries into
//            the population's region of a shared-memory stage, completing on
//            the stage's mbarrier;
//   * update: each thread takes node pairs of the band, reads the pair's slots
//            from shared memory, collides in packed FP32x2 and writes the
//            results back to the same shared-memory slots;
//   * store: one bulk copy of the span's 16-byte-aligned interior back to
//            global memory; the few elements of the span in its first and last
//            16-byte chunk (which it shares with neighbouring spans) are stored
//            one by one, so that no other band's slots are overwritten.
// The first and the last row of every run are bands of their own, so that no
// span wraps around the periodic y boundary: rows 0 and ny - 1 read, in the odd
// sweep, the single rows ny - 1 and 0 (e_y = -1 and +1), and the bands in
// between stay inside 1 .. ny - 2 with their neighbour rows.
//
// Pairs.  Even nx: x-neighbour pairs as in the single-grid pair sweep ((x0,
// x0 + 1) with x0 even in the even sweep, x0 odd in the odd sweep, so that the
// 2-element slots of e_x = +-1 are aligned and only e_x = 0 needs two
// 1-element accesses; spans of even-nx runs start at even elements).  Odd nx:
// consecutive nodes of the band in row-major order, each lane with its own
// 1-element accesses; an odd node count leaves lane 1 of the last pair
// repeating lane 0's node (same slots, same values).
//
// Pipeline.  kStages shared-memory stages per CTA; one producer warp and
// kConsumers / 32 consumer warps, synchronised only through mbarriers.  The
// producer starts the loads of a stage's band (full[s]: one arrival carrying
// the byte count), the consumers update it and arrive on done[s] (one arrival
// per warp, after a proxy fence), then the producer stores the band and
// reloads the stage with the band kStages further on.  While the consumers
// update band i, the loads of bands i + 1 .. i + kStages - 1 are in flight.
// Every mbarrier wait is bounded: a wait that gives up sets bit 2 of the run's
// status word; the producer then waits (bounded again) for the copies it
// started before the CTA returns.
#pragma once

#include "sweep_body.cuh"
#include "tc05.cuh"

namespace lbm {
namespace stg {

constexpr int kHdrBytes = 192;
constexpr int kBarBytes = 128;  // up to 8 stages: full[] and done[] mbarriers
constexpr int kWaitPolls = 1 << 20;
constexpr int kMaxNx = 4096;  // widest run row the staged sweep takes (also bounded by the band capacity)

// Launch shape: consumer threads, stages, band bytes per population, CTAs per SM.
// A stage is reloaded as soon as its band's bulk store has read it.
template <int CONS, int STAGES, int SPAN, int MINB>
struct Cfg {
  static constexpr int kConsumers = CONS;
  static constexpr int kThreads = CONS + 32;  // plus the producer warp
  static constexpr int kStages = STAGES;
  static constexpr int kSpanBytes = SPAN;
  static constexpr int kMinBlocks = MINB;
  static constexpr int kRegionBytes = SPAN + 32;  // plus the rounding to 16-byte chunks
  static constexpr int kStageBytes = kHdrBytes + 9 * kRegionBytes;
  static constexpr int kSmemBytes = kBarBytes + STAGES * kStageBytes;
  static_assert(2 * STAGES * 8 <= kBarBytes, "mbarrier area too small");
  static_assert(STAGES >= 2, "a band in flight while another is updated");
};

template <int S>
__host__ __device__ constexpr int elem_bytes() {
  return S == LBM_F32 ? 4 : 2;
}

// floor(p / d) = high word of p * m with m = ceil(2^32 / d), exact for p, d < 2^16
// (the error p (m - 2^32 / d) / 2^32 stays below 1 / d); m = 0 stands for d = 1.
inline uint32_t div_magic(uint32_t d) { return d <= 1 ? 0u : (uint32_t)((((uint64_t)1 << 32) + d - 1) / d); }
__device__ __forceinline__ uint32_t div_small(uint32_t p, uint32_t m) { return m ? __umulhi(p, m) : p; }

struct Band {
  int run, y0, rows, pad;
};

// Written by the issuing thread before the stage's mbarrier arrive (release),
// read by every thread after its wait (acquire).
struct Hdr {
  int64_t g0[9];  // population-buffer element index of population j's span start
  int run, y0, rows, skip;
  uint32_t nx, ny, m_nx, m_half;
  int sh[9];  // element offset of population j's band row 0 in its region
  float om[5];
};
static_assert(sizeof(Hdr) <= kHdrBytes, "stage header too large");

__device__ __forceinline__ void arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc05::smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc05::smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          tc05::smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(tc05::smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void bulk_store(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(tc05::smem_u32(src)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// wait until at most N committed store groups still read shared memory
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

template <class C>
__device__ __forceinline__ unsigned char* region(unsigned char* st, int j) {
  return st + kHdrBytes + j * C::kRegionBytes;
}

// Producer warp: fill the header of stage `st` for band `bd` and start its
// copies; lane j < 9 takes population j's span.
template <class C, int S, bool ODD, class Run>
__device__ __forceinline__ void issue(unsigned char* st, uint64_t* bar, const typename PairIO<S>::E* f,
                                      const Run* runs, const Band& bd, const int* status, int lane) {
  constexpr int esz = elem_bytes<S>(), epc = 16 / esz;
  Hdr* h = reinterpret_cast<Hdr*>(st);
  const Run& R = runs[bd.run];
  const int64_t nx = R.nx, ny = R.ny, N = nx * ny;
  const int skip = status[bd.run] != 0;
  if (lane == 0) {
    h->run = bd.run;
    h->y0 = bd.y0;
    h->rows = bd.rows;
    h->nx = (uint32_t)nx;
    h->ny = (uint32_t)ny;
    h->m_nx = R.m_nx;
    h->m_half = R.m_half;
    h->skip = skip;
  }
  if (lane < 5) h->om[lane] = (float)R.om[lane];
  int64_t a0 = 0;
  uint32_t bytes = 0;
  if (lane < 9) {
    const int j = lane;
    const int ey = ODD ? j / 3 - 1 : 0;  // e_y of velocity j (j = (e_x + 1) + 3 (e_y + 1))
    int64_t r0 = bd.y0 + ey;             // wraps only for the one-row bands at y = 0 and y = ny - 1
    r0 = r0 < 0 ? r0 + ny : (r0 >= ny ? r0 - ny : r0);
    const int64_t g0 = R.off + j * N + r0 * nx;
    const int64_t g1 = g0 + bd.rows * nx;
    a0 = g0 & ~(int64_t)(epc - 1);
    const int64_t a1 = (g1 + epc - 1) & ~(int64_t)(epc - 1);
    h->sh[j] = (int)(g0 - a0);
    h->g0[j] = g0;
    bytes = (uint32_t)((a1 - a0) * esz);
  }
  const uint32_t total = __reduce_add_sync(0xffffffffu, bytes);
  if (lane == 0) {
    if (skip)
      arrive(bar);
    else
      arrive_expect_tx(bar, total);
  }
  __syncwarp();
  if (!skip && lane < 9) bulk_load(region<C>(st, lane), f + a0, bytes, bar);
}

// Node pairs of the band, updated in shared memory.  Returns false when a node is unphysical.
template <class C, int S, bool ODD>
__device__ __forceinline__ bool update_band(unsigned char* st, const Hdr& h) {
  using IO = PairIO<S>;
  using E = typename IO::E;
  const uint32_t nx = h.nx;
  f2 om[5];
#pragma unroll
  for (int n = 0; n < 5; ++n) om[n] = pack2(h.om[n], h.om[n]);
  E* reg[9];  // span j's band-row-0 element in shared memory
#pragma unroll
  for (int j = 0; j < 9; ++j) reg[j] = reinterpret_cast<E*>(region<C>(st, j)) + h.sh[j];
  auto out = [&](int j, uint32_t m) -> E* { return reg[j] + m; };  // results go back to the same slots
  bool ok = true;
  if ((nx & 1u) == 0) {
    const uint32_t half = nx >> 1, np = (uint32_t)h.rows * half;
    for (uint32_t p = threadIdx.x; p < np; p += C::kConsumers) {
      // even sweep: the pair's slots are band elements 2p, 2p + 1 (row + x0 = 2p)
      const uint32_t k = ODD ? div_small(p, h.m_half) : 0u, xp = p - k * half;
      const uint32_t row = k * nx;
      const uint32_t x0 = 2 * xp + (ODD ? 1u : 0u);
      const uint32_t x1 = x0 + 1 == nx ? 0u : x0 + 1;
      RawPair r[9];
#pragma unroll
      for (int j = 0; j < 9; ++j) {
        const int dx = tp::dig(j, 0);
        E* b = reg[j] + row;
        if (!ODD)
          IO::raw2(b + x0, r[j]);
        else if (dx == 1)
          IO::raw11(b + x0, b + x1, r[j]);
        else
          IO::raw2(b + (dx == 0 ? x0 - 1 : x1), r[j]);
      }
      f2 v[9];
      tp::pair_decode<2, S, ODD>(r, v);
      ok = tp::collide<f2, 2>(v, om) && ok;
#pragma unroll
      for (int j = 0; j < 9; ++j) {
        const int dx = tp::dig(j, 0);
        f2 val = ODD ? v[j] : v[tp::opp<2>(j)];
        if (IO::kScaled) val = val * cst<f2>(tp::iwq<2>(j));
        if (!ODD)
          IO::store2(out(j, row + x0), val);
        else if (dx == 1)
          IO::store11(out(j, row + x0), out(j, row + x1), val);
        else
          IO::store2(out(j, row + (dx == 0 ? x0 - 1 : x1)), val);
      }
    }
  } else {
    const uint32_t n = (uint32_t)h.rows * nx, np = (n + 1) >> 1;
    for (uint32_t p = threadIdx.x; p < np; p += C::kConsumers) {
      const uint32_t n0 = 2 * p;
      // slot offsets of lane 0 / lane 1 for e_x = -1, 0, +1 (row of the band's span, shifted column);
      // the even sweep reads the nodes' own slots, band elements n0 and n0 + 1
      uint32_t la[3], lb[3];
      la[1] = n0;
      lb[1] = n0 + 1 < n ? n0 + 1 : n0;
      if (ODD) {
        const uint32_t k0 = div_small(n0, h.m_nx), xa = n0 - k0 * nx;
        uint32_t k1 = k0, xb = xa;
        if (n0 + 1 < n) {
          xb = xa + 1;
          if (xb == nx) {
            xb = 0;
            k1 = k0 + 1;
          }
        }
        la[0] = k0 * nx + (xa == 0 ? nx - 1 : xa - 1);
        la[2] = k0 * nx + (xa + 1 == nx ? 0 : xa + 1);
        lb[0] = k1 * nx + (xb == 0 ? nx - 1 : xb - 1);
        lb[2] = k1 * nx + (xb + 1 == nx ? 0 : xb + 1);
      }
      RawPair r[9];
#pragma unroll
      for (int j = 0; j < 9; ++j) {
        const int dx = ODD ? tp::dig(j, 0) : 1;
        IO::raw11(reg[j] + la[dx], reg[j] + lb[dx], r[j]);
      }
      f2 v[9];
      tp::ypair_decode<S, ODD>(r, v);
      ok = tp::collide<f2, 2>(v, om) && ok;
#pragma unroll
      for (int j = 0; j < 9; ++j) {
        const int dx = ODD ? tp::dig(j, 0) : 1;
        f2 val = ODD ? v[j] : v[tp::opp<2>(j)];
        if (IO::kScaled) val = val * cst<f2>(tp::iwq<2>(j));
        IO::store11(out(j, la[dx]), out(j, lb[dx]), val);
      }
    }
  }
  return ok;
}

// Producer warp: lane j < 9 stores population j's span: its 16-byte-aligned
// interior by one bulk copy (one commit group per lane and band), and lanes
// j and j + 9 the elements before and after it one by one (at most 7 each;
// those chunks are shared with neighbouring spans).
template <class C, int S>
__device__ __forceinline__ void store_band(unsigned char* st, typename PairIO<S>::E* f, const Hdr& h, int lane) {
  using E = typename PairIO<S>::E;
  constexpr int esz = elem_bytes<S>(), epc = 16 / esz;
  if (lane >= 18) return;
  const int j = lane < 9 ? lane : lane - 9;
  const int64_t len = (int64_t)h.rows * h.nx;
  const int64_t g0 = h.g0[j], g1 = g0 + len;
  const int64_t c0 = (g0 + epc - 1) & ~(int64_t)(epc - 1), c1 = g1 & ~(int64_t)(epc - 1);
  const E* reg = reinterpret_cast<const E*>(region<C>(st, j)) + h.sh[j];
  if (lane < 9) {
    if (c1 > c0) bulk_store(f + c0, reg + (c0 - g0), (uint32_t)((c1 - c0) * esz));
    bulk_commit();
    // elements before the interior (the whole span when it has none)
    const int64_t e1 = c1 > c0 ? c0 : g1;
    for (int64_t g = g0; g < e1; ++g) f[g] = reg[g - g0];
  } else if (c1 > c0) {
    for (int64_t g = c1; g < g1; ++g) f[g] = reg[g - g0];
  }
}

template <class C, int S, bool ODD, class Run>
__global__ void __launch_bounds__(C::kThreads, C::kMinBlocks)
    staged_kernel(typename PairIO<S>::E* __restrict__ f, const Run* __restrict__ runs, const Band* __restrict__ bands,
                  int nbands, int* __restrict__ status) {
  constexpr int NS = C::kStages;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* done = full + NS;
  unsigned char* stages = smem + kBarBytes;
  const int tid = threadIdx.x, lane = tid & 31;
  const int mine = (int)blockIdx.x < nbands ? (nbands - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      tc05::mbar_init(&full[s], 1);
      tc05::mbar_init(&done[s], C::kConsumers / 32);
    }
    fence_barrier_init();
  }
  __syncthreads();
  if (tid >= C::kConsumers) {
    // producer warp
    int filled = 0, i = 0, bad = 0;
    for (; filled < NS && filled < mine; ++filled)
      issue<C, S, ODD>(stages + filled * C::kStageBytes, &full[filled], f, runs,
                       bands[blockIdx.x + filled * gridDim.x], status, lane);
    for (; i < mine; ++i) {
      const int s = i % NS;
      unsigned char* st = stages + s * C::kStageBytes;
      if (!tc05::mbar_wait(&done[s], (uint32_t)((i / NS) & 1), kWaitPolls)) {
        bad = 1;
        break;
      }
      const Hdr& h = *reinterpret_cast<const Hdr*>(st);
      if (!h.skip)
        store_band<C, S>(st, f, h, lane);
      else if (lane < 9)
        bulk_commit();  // an empty group keeps one group per lane and band
      // reload this stage with the band NS further on, once its store has read it
      if (filled < mine) {
        if (lane < 9) bulk_wait_read<0>();
        __syncwarp();
        issue<C, S, ODD>(st, &full[s], f, runs, bands[blockIdx.x + filled * gridDim.x], status, lane);
        ++filled;
      }
    }
    if (lane < 9) bulk_wait_all();
    if (bad && lane == 0) {
      const Hdr& h = *reinterpret_cast<const Hdr*>(stages + (i % NS) * C::kStageBytes);
      atomicOr(&status[h.run], 2);
      // let the loads already started land before the CTA returns
      for (int k = i; k < filled; ++k) tc05::mbar_wait(&full[k % NS], (uint32_t)((k / NS) & 1), kWaitPolls);
    }
    return;
  }
  // consumer warps
  for (int i = 0; i < mine; ++i) {
    const int s = i % NS;
    unsigned char* st = stages + s * C::kStageBytes;
    if (!tc05::mbar_wait(&full[s], (uint32_t)((i / NS) & 1), kWaitPolls)) {
      if (lane == 0) atomicOr(&status[reinterpret_cast<const Hdr*>(st)->run], 2);
      break;
    }
    const Hdr& h = *reinterpret_cast<const Hdr*>(st);
    if (!h.skip) {
      if (!update_band<C, S, ODD>(st, h)) atomicOr(&status[h.run], 1);
      tc05::fence_proxy_async();  // this thread's shared-memory results, before the bulk store reads them
    }
    __syncwarp();
    if (lane == 0) arrive(&done[s]);
  }
}

// The launch shapes the batch chooses from (variant k = index k).
using V0 = Cfg<256, 2, 6144, 2>;
using V1 = Cfg<256, 3, 4096, 2>;
using V2 = Cfg<512, 2, 12288, 1>;
using V3 = Cfg<512, 3, 8192, 1>;
constexpr int kVariants = 4;
// nodes per band at most (host side: the band lists)
inline int capacity(int variant, int esz) {
  const int span[kVariants] = {V0::kSpanBytes, V1::kSpanBytes, V2::kSpanBytes, V3::kSpanBytes};
  return span[variant] / esz;
}

}  // namespace stg
}  // namespace lbm
