// Front Schur update on the 5th-generation tensor cores (sm_103a):
//     C[kend:, kend:] -= W L^T      (lower triangle, FP32 fronts)
// where W = L21 D and L = L21 of one outer block (inner dimension <= 256).
//
// The output is cut into 128-row units, each accumulated by one CTA: one
// 128 x 128 tile, or two tiles of the same tile row side by side (128 x 256,
// one N = 256 MMA), which share the W operand and so cut the operand bytes
// per output entry by a quarter.
// W and L are kept in K-major global arrays split as x = hi + lo with hi = x
// with its low 13 mantissa bits cleared (exactly representable in TF32) and
// lo = x - hi; the unit is accumulated in TMEM (FP32) as
// Whi Lhi^T + Whi Llo^T + Wlo Lhi^T ("3xTF32"), which keeps FP32-level
// accuracy on the TF32 tensor path.
//
// Every mbarrier wait is bounded; on expiry the CTA records DEV_TIMEOUT in
// the status word, drains the copies it issued (bounded again), frees its
// TMEM and returns.
#pragma once

#include <cuda.h>
#include <cstdint>

namespace sgn {
namespace tc {

constexpr int TILE = 128;          // output tile (M = N)
constexpr int KCH = 32;            // K per stage: 32 FP32 = one 128-byte swizzle row
constexpr int TILE_BYTES = TILE * KCH * 4;           // 16 KB
// operand stages: single-tile units stage Whi, Wlo, Lhi, Llo (64 KB, three
// stages); pair units Whi, Wlo, Lhi x 2, Llo x 2 (96 KB, two stages)
template <bool PAIR> struct Stages {
  static constexpr int N = PAIR ? 2 : 3;
  static constexpr int BYTES = (PAIR ? 6 : 4) * TILE_BYTES;
  static constexpr int LLO = PAIR ? 4 : 3;  // tile slot of Llo
};
constexpr long long WAIT_CYCLES = 1ll << 31;         // ~1 s at 2 GHz

struct Maps {                      // one set of tensor maps per front
  CUtensorMap whi, wlo, lhi, llo;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait: false (and DEV_TIMEOUT recorded) if the phase never completes
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *status, int flag) {
  long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > WAIT_CYCLES) {
      atomicOr(status, flag);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(smem_u32(bar))
      : "memory");
}

// UMMA shared-memory descriptor: K-major operand, 128B swizzle, 8-row
// groups 1024 bytes apart (SBO), descriptor version 1
__device__ __forceinline__ uint64_t umma_desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)(16 >> 4) << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// instruction descriptor: D FP32, A and B TF32, both K-major, M = 128, N = n
__host__ __device__ constexpr uint32_t idesc_tf32_128xn(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TILE >> 4) << 24);
}

__device__ __forceinline__ void umma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld_32x32b_x32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld_32x32b_x16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// the hi / lo split used for the 3xTF32 products
__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// ---------------------------------------------------------------------------
// Persistent, warp-specialised trailing update: each CTA walks its share of
// one flat list of units over every front of a level (units first, first +
// stride, ...); two TMEM accumulators (2 x 256 columns) let the epilogue of
// unit i run while the producer and MMA warps already work on unit i + 1.
// The unit source maps a list index to its front's job, tensor maps and the
// unit's index in that front's window (Src::get); every role walks the same
// sequence.
//   warp 0 lane 0 : TMA producer      warp 1 lane 0 : MMA issuer (+ TMEM alloc)
//   warps 2..9    : epilogue (warp w reads TMEM lanes 32 (w % 4) .. + 31 and
//                   half of the unit's columns, (w - 2) / 4 naming the half)
constexpr int PTHREADS = 320;
constexpr int EPI_WARPS = 8;
constexpr int PSMEM_BYTES = (Stages<true>::N * Stages<true>::BYTES > Stages<false>::N * Stages<false>::BYTES
                                 ? Stages<true>::N * Stages<true>::BYTES
                                 : Stages<false>::N * Stages<false>::BYTES) +
                            1024;  // + alignment slack

struct TileJob {                 // one front's part of a trailing update
  float *L;                      // the front's factor columns (f x ns, column-major)
  float *CB;                     // its contribution block ((f - ns) x (f - ns))
  int64_t f, ns;
  int nrows;                     // f - kend
  int kend;                      // first trailing row (TMA row coordinate of tile row 0)
  int kchunks;                   // 32-wide K chunks
  int ntiles;                    // units of the window
  int win0, m;                   // the window: tile columns win0 .. win0 + m - 1 (rows >= columns)
  int pair;                      // units are tile pairs (else single tiles)
};

// Units of a window of m tile columns over n tile rows (rows >= columns
// within the window's m x m triangle, then n - m full rows).  Single tiles:
// m (m + 1) / 2 + (n - m) m.  Pairs (tile columns 2u, 2u + 1 of one tile row,
// the last one of a row single when the row has an odd number of tiles):
// triangle row r holds floor(r / 2) + 1 units, a full row ceil(m / 2).
__host__ __device__ __forceinline__ int window_units(int m, int n, bool pair) {
  if (m <= 0) return 0;
  if (!pair) return m * (m + 1) / 2 + (n - m) * m;
  const int q = m / 2;
  const int tri = (m & 1) ? (q + 1) * (q + 1) : q * (q + 1);
  return tri + (n - m) * ((m + 1) / 2);
}

__host__ __device__ __forceinline__ void tile_coords(int tile, int &bi, int &bj) {
  bi = (int)((sqrtf(8.f * (float)tile + 1.f) - 1.f) * 0.5f);  // corrected below
  while ((bi + 1) * (bi + 2) / 2 <= tile) ++bi;
  while (bi * (bi + 1) / 2 > tile) --bi;
  bj = tile - bi * (bi + 1) / 2;
}

// unit t of a job's window, row-major: the window's triangle first, then its
// rows below.  (bi, bj) is the unit's first tile (absolute tile coordinates,
// bi >= bj); two = the unit also holds tile (bi, bj + 1)
__host__ __device__ __forceinline__ void window_unit(const TileJob &job, int t, int &bi, int &bj, bool &two) {
  int r, c;
  if (!job.pair) {
    const int t0 = job.m * (job.m + 1) / 2;
    if (t < t0) {
      tile_coords(t, r, c);
    } else {
      r = job.m + (t - t0) / job.m;
      c = (t - t0) % job.m;
    }
    two = false;
  } else {
    const int t0 = window_units(job.m, job.m, true);
    if (t < t0) {
      // triangle rows 2q and 2q + 1 hold q + 1 units each: units q (q + 1) ..
      int q = (int)((sqrtf(4.f * (float)t + 1.f) - 1.f) * 0.5f);  // corrected below
      while ((q + 1) * (q + 2) <= t) ++q;
      while (q * (q + 1) > t) --q;
      const int o = t - q * (q + 1);
      r = o <= q ? 2 * q : 2 * q + 1;
      c = 2 * (o <= q ? o : o - q - 1);
      two = c + 1 <= r;
    } else {
      const int per = (job.m + 1) / 2;
      r = job.m + (t - t0) / per;
      c = 2 * ((t - t0) % per);
      two = c + 1 < job.m;
    }
  }
  bi = job.win0 + r;
  bj = job.win0 + c;
}

template <bool PAIR, typename Src>
__device__ __forceinline__ void tile_loop_tc(const Src &src, int ntiles, int first, int stride, int *status,
                                             int flag_timeout) {
  extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
  constexpr int PSTAGES = Stages<PAIR>::N, STAGE_BYTES = Stages<PAIR>::BYTES, LLO = Stages<PAIR>::LLO;
  __shared__ uint64_t full_bar[PSTAGES], empty_bar[PSTAGES], acc_full[2], acc_empty[2];
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  unsigned char *sm = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int my_tiles = first < ntiles ? (ntiles - first + stride - 1) / stride : 0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < PSTAGES; ++s) { mbar_init(&full_bar[s], 1); mbar_init(&empty_bar[s], 1); }
    for (int b = 0; b < 2; ++b) { mbar_init(&acc_full[b], 1); mbar_init(&acc_empty[b], EPI_WARPS); }
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(4 * TILE)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  // stage layout of a pair list: Whi | Wlo | Lhi (tile bj) | Lhi (tile bj + 1)
  // | Llo (bj) | Llo (bj + 1): the two L tiles of a pair sit back to back, so
  // that one K-major 256-row operand (8-row groups 1 KB apart) covers both;
  // of a single-tile list: Whi | Wlo | Lhi | Llo
  if (warp == 0) {
    if (lane == 0 && my_tiles > 0) {
      const Maps *cur = nullptr;
      int g = 0;  // global chunk counter over all of this CTA's units
      bool stop = false;
      for (int lt = 0; lt < my_tiles && !stop; ++lt) {
        TileJob job;
        const Maps *maps;
        int t;
        src.get(first + lt * stride, job, maps, t);
        if (maps != cur) {
          asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&maps->whi) : "memory");
          asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&maps->wlo) : "memory");
          asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&maps->lhi) : "memory");
          asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&maps->llo) : "memory");
          cur = maps;
        }
        int bi, bj;
        bool two;
        window_unit(job, t, bi, bj, two);
        const int rw = job.kend + bi * TILE, rl = job.kend + bj * TILE;
        for (int kc = 0; kc < job.kchunks; ++kc, ++g) {
          const int s = g % PSTAGES;
          if (g >= PSTAGES && !mbar_wait(&empty_bar[s], ((g / PSTAGES) - 1) & 1, status, flag_timeout)) {
            abort_flag = 1; stop = true; break;
          }
          if (*(volatile int *)&abort_flag) { stop = true; break; }
          unsigned char *st = sm + s * STAGE_BYTES;
          mbar_expect_tx(&full_bar[s], (two ? 6 : 4) * TILE_BYTES);
          tma_load_2d(st + 0 * TILE_BYTES, &maps->whi, &full_bar[s], kc * KCH, rw);
          tma_load_2d(st + 1 * TILE_BYTES, &maps->wlo, &full_bar[s], kc * KCH, rw);
          tma_load_2d(st + 2 * TILE_BYTES, &maps->lhi, &full_bar[s], kc * KCH, rl);
          tma_load_2d(st + LLO * TILE_BYTES, &maps->llo, &full_bar[s], kc * KCH, rl);
          if (PAIR && two) {
            tma_load_2d(st + 3 * TILE_BYTES, &maps->lhi, &full_bar[s], kc * KCH, rl + TILE);
            tma_load_2d(st + 5 * TILE_BYTES, &maps->llo, &full_bar[s], kc * KCH, rl + TILE);
          }
        }
      }
      // drain the copies still in flight (bounded)
      for (int q = (g > PSTAGES ? g - PSTAGES : 0); q < g; ++q)
        mbar_wait(&full_bar[q % PSTAGES], (q / PSTAGES) & 1, status, flag_timeout);
    }
  } else if (warp == 1) {
    if (lane == 0 && my_tiles > 0) {
      int g = 0;
      bool stop = false;
      for (int lt = 0; lt < my_tiles && !stop; ++lt) {
        TileJob job;
        const Maps *maps;
        int t;
        src.get(first + lt * stride, job, maps, t);
        int bi, bj;
        bool two;
        window_unit(job, t, bi, bj, two);
        const uint32_t idesc = idesc_tf32_128xn(two ? 2 * TILE : TILE);
        const int kch = job.kchunks;
        const int b = lt & 1;
        if (lt >= 2 && !mbar_wait(&acc_empty[b], ((lt >> 1) - 1) & 1, status, flag_timeout)) {
          abort_flag = 1; break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t acc_tmem = tmem + (uint32_t)(b * 2 * TILE);
        for (int kc = 0; kc < kch; ++kc, ++g) {
          const int s = g % PSTAGES;
          if (!mbar_wait(&full_bar[s], (g / PSTAGES) & 1, status, flag_timeout)) { abort_flag = 1; stop = true; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t base = smem_u32(sm + s * STAGE_BYTES);
#pragma unroll
          for (int k = 0; k < KCH / 8; ++k) {
            const uint32_t off = k * 32;
            const uint64_t ahi = umma_desc_sw128(base + 0 * TILE_BYTES + off);
            const uint64_t alo = umma_desc_sw128(base + 1 * TILE_BYTES + off);
            const uint64_t bhi = umma_desc_sw128(base + 2 * TILE_BYTES + off);
            const uint64_t blo = umma_desc_sw128(base + LLO * TILE_BYTES + off);
            umma_tf32(acc_tmem, ahi, bhi, idesc, (kc | k) != 0);
            umma_tf32(acc_tmem, ahi, blo, idesc, 1);
            umma_tf32(acc_tmem, alo, bhi, idesc, 1);
          }
          umma_commit(&empty_bar[s]);
        }
        if (stop) break;
        umma_commit(&acc_full[b]);
      }
      if (*(volatile int *)&abort_flag) {
        // release the epilogue of both buffers so nobody waits for a full second
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc_full[0])) : "memory");
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc_full[1])) : "memory");
      }
    }
  } else {
    // epilogue warps 2..9: a quarter of the unit's rows (TMEM lanes) and
    // half of its columns each (64 of a single-tile list's tiles, 128 of a
    // pair list's units)
    const int quad = warp & 3;
    const int half = (warp - 2) / 4;
    const int r = quad * 32 + lane;
    for (int lt = 0; lt < my_tiles; ++lt) {
      const int b = lt & 1;
      // the unit and its C entries do not depend on the accumulator: the
      // warp's columns go in 16-column chunks, the first two loaded before
      // the wait and each later one while an earlier one is written, so
      // that the loads' latency overlaps the MMAs
      TileJob job;
      const Maps *maps;
      int t;
      src.get(first + lt * stride, job, maps, t);
      int bi, bj;
      bool two;
      window_unit(job, t, bi, bj, two);
      const int wcols = job.pair ? TILE : TILE / 2;  // this warp's column span
      const int col0 = half * wcols;
      const int nch = wcols / 16;
      const int rows = min(TILE, job.nrows - bi * TILE);
      const int cols = min(two ? 2 * TILE : TILE, job.nrows - bj * TILE);
      const bool active = col0 < cols;  // warp-uniform
      const int roff = (bi - bj) * TILE;
      // element (gi, gj) of the front: factor column (gj < ns) or
      // contribution block (gj >= ns, then gi >= gj >= ns)
      const int64_t gi = (int64_t)job.kend + bi * TILE + r, gj0 = (int64_t)job.kend + bj * TILE;
      const int64_t fcb = job.f - job.ns;
      auto elem = [&](int cc) -> float * {
        const int64_t gj = gj0 + cc;
        return gj < job.ns ? job.L + gi + gj * job.f : job.CB + (gi - job.ns) + (gj - job.ns) * fcb;
      };
      // the 16 entries of chunk cb of this thread's row: in one region (one
      // base pointer, one stride), or, for a chunk that straddles the last
      // factor column ns, element by element.  C is touched once per outer
      // block: streaming loads and stores (evict first), so that L2 keeps the
      // operand tiles that other units reuse
      auto load_chunk = [&](int cb, float (&cv)[16]) {
        if (r >= rows) return;
        const int64_t gjc = gj0 + cb;
        if (gjc + 15 < job.ns || gjc >= job.ns) {
          const bool in_l = gjc < job.ns;
          const float *__restrict__ base = in_l ? job.L + gi + gjc * job.f : job.CB + (gi - job.ns) + (gjc - job.ns) * fcb;
          const int64_t st = in_l ? job.f : fcb;
#pragma unroll
          for (int j = 0; j < 16; ++j) cv[j] = (cb + j < cols && r + roff >= cb + j) ? __ldcs(base + j * st) : 0.f;
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) cv[j] = (cb + j < cols && r + roff >= cb + j) ? __ldcs(elem(cb + j)) : 0.f;
        }
      };
      auto store_chunk = [&](int cb, const float (&cv)[16], const uint32_t (&v)[16]) {
        if (r >= rows) return;
        const int64_t gjc = gj0 + cb;
        if (gjc + 15 < job.ns || gjc >= job.ns) {
          const bool in_l = gjc < job.ns;
          float *__restrict__ base = in_l ? job.L + gi + gjc * job.f : job.CB + (gi - job.ns) + (gjc - job.ns) * fcb;
          const int64_t st = in_l ? job.f : fcb;
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (cb + j < cols && r + roff >= cb + j) __stcs(base + j * st, cv[j] - __uint_as_float(v[j]));
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (cb + j < cols && r + roff >= cb + j) __stcs(elem(cb + j), cv[j] - __uint_as_float(v[j]));
        }
      };
      float ca[16], cb2[16];
      if (active) {
        load_chunk(col0, ca);
        load_chunk(col0 + 16, cb2);
      }
      bool ok = mbar_wait(&acc_full[b], (lt >> 1) & 1, status, flag_timeout);
      // tcgen05.ld is warp-collective: the whole warp takes the same branch
      ok = __all_sync(0xffffffffu, ok && !*(volatile int *)&abort_flag);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (!ok) break;
      if (active) {
        uint32_t v[16];
        const uint32_t trow = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(b * 2 * TILE + col0);
        for (int q = 0; q < nch; q += 2) {
          tmem_ld_32x32b_x16(trow + 16u * q, v);
          store_chunk(col0 + 16 * q, ca, v);
          if (q + 2 < nch) load_chunk(col0 + 16 * (q + 2), ca);
          tmem_ld_32x32b_x16(trow + 16u * (q + 1), v);
          store_chunk(col0 + 16 * (q + 1), cb2, v);
          if (q + 3 < nch) load_chunk(col0 + 16 * (q + 3), cb2);
        }
      }
      // this warp's TMEM reads of buffer b are complete (tcgen05.wait::ld)
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc_empty[b])) : "memory");
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(4 * TILE) : "memory");
  }
}

}  // namespace tc
}  // namespace sgn
