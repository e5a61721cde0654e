// tile2d.cuh -- device code of the planar bit-sliced tile kernels: the
// one-instance step (step_tiled.cu) and the batched step (batch_kernels.cu)
// are instantiated from these templates in two translation units, so that
// they compile in parallel.  The design is described in step_tiled.cu.
#pragma once

#include <stdint.h>

#include "bitslice.cuh"
#include "squeeze_internal.cuh"

namespace sq {
namespace {

constexpr int kTiledMaxThreads = 384;
constexpr uint32_t kTiledPasses = 8;            // most steps per launch the handle's program is built for
constexpr size_t kTiledSmemCap = 56 * 1024;     // default level: 4 CTAs per SM
constexpr size_t kTiledSmemLimit = 200 * 1024;  // any level: one CTA per SM

__device__ __forceinline__ void flag(int *status, int code) { atomicCAS(status, 0, code); }

// Outer-totalistic rule on 32 cells at once: n[0..7] are the neighbour bits.
// kLife: the rule is B3/S23, evaluated as "count in {2,3} and (count odd or
// alive)"; otherwise the birth/survive masks are evaluated count by count.
template <bool kLife>
__device__ __forceinline__ uint32_t rule_word(const Rule &rule, uint32_t self, const uint32_t *n) {
  uint32_t s0 = n[0] ^ n[1] ^ n[2], c0 = maj3(n[0], n[1], n[2]);
  uint32_t s1 = n[3] ^ n[4] ^ n[5], c1 = maj3(n[3], n[4], n[5]);
  uint32_t s2 = n[6] ^ n[7], c2 = n[6] & n[7];
  uint32_t b0 = s0 ^ s1 ^ s2, c3 = maj3(s0, s1, s2);
  uint32_t t = c0 ^ c1 ^ c2, u = maj3(c0, c1, c2);
  uint32_t b1 = t ^ c3, v = t & c3;
  uint32_t b2 = u ^ v, b3 = u & v;
  if (kLife) return b1 & ~b2 & ~b3 & (b0 | self);
  uint32_t next = 0, any = rule.birth | rule.survive;
#pragma unroll
  for (uint32_t c = 0; c <= 8; ++c) {
    if (!((any >> c) & 1u)) continue;
    uint32_t e = ((c & 1u) ? b0 : ~b0) & ((c & 2u) ? b1 : ~b1) & ((c & 4u) ? b2 : ~b2) &
                 ((c & 8u) ? b3 : ~b3);
    bool bb = (rule.birth >> c) & 1u, ss = (rule.survive >> c) & 1u;
    next |= bb && ss ? e : (bb ? (e & ~self) : (e & self));
  }
  return next;
}

// Carry walk: the level-L block adjacent to tile (tx, ty) in direction
// (dx, dy), as a tile (ntx, nty), or false for a hole / off the box.  Tile
// coordinates fit 32 bits, so the digit updates use wrap-around arithmetic.
// Host-callable too, so that the walk can be checked on the CPU.
__host__ __device__ bool adjacent_tile(const FracDev &f, uint32_t L, const uint8_t *taux,
                              const uint8_t *tauy, const uint8_t *hnu, uint32_t tx, uint32_t ty,
                              int dx, int dy, uint32_t &ntx, uint32_t &nty) {
  int cx = dx, cy = dy;
  uint32_t qx = tx, qy = ty, pwx = 1, pwy = 1, ax = tx, ay = ty;
  for (uint32_t mu = L + 1; mu <= f.r && (cx | cy); ++mu) {
    bool odd = mu & 1u;
    uint32_t src = odd ? qx : qy;
    uint32_t q = fdiv(f.divk, src);
    uint32_t beta = src - q * f.k;
    int ox = (int)taux[beta] + cx, oy = (int)tauy[beta] + cy;
    cx = ox < 0 ? -1 : (ox >= (int)f.s ? 1 : 0);
    cy = oy < 0 ? -1 : (oy >= (int)f.s ? 1 : 0);
    ox -= cx * (int)f.s;
    oy -= cy * (int)f.s;
    uint32_t nb = hnu[oy * f.s + ox];
    if (nb == kHole) return false;
    uint32_t delta = nb - beta;
    if (odd) {
      qx = q;
      ax += delta * pwx;
      pwx *= f.k;
    } else {
      qy = q;
      ay += delta * pwy;
      pwy *= f.k;
    }
  }
  if (cx | cy) return false;  // carried past the top level: off the box
  ntx = ax;
  nty = ay;
  return true;
}

// ---- bulk asynchronous copies (TMA, non-tensor form) and mbarriers ----------

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *m, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(m)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *m, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(m)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait_at(uint32_t addr, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(addr), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *m, uint32_t parity) {
  return mbar_try_wait_at(smem_u32(m), parity);
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Abort record of the CTA: set by the first wait that gives up, with the
// shared-memory address of the barrier and the phase it gave up on, the wait
// limit, the status word to report to, and whether any copy was issued at
// all (not under the load-withholding test hook).
struct AbortRecord {
  uint32_t bar;
  uint32_t parity;
  uint32_t set;
  uint32_t nocopy;
  uint64_t limit;
  int *status;
};
__shared__ AbortRecord g_abort;

// Wait for an mbarrier phase, giving up after `limit` ns (2 s unless the
// handle sets another) with DEVICE_TIMEOUT.  A wait that gives up records it
// in g_abort; every later wait of the CTA that does not complete at once
// returns as soon as it sees the record, and no more loads are issued, so a
// copy that never lands costs the launch one limit instead of one per group.
// Control flow is unchanged (every thread still reaches every barrier); the
// results of an aborted launch are not valid, which the status word says.
__device__ __noinline__ void mbar_wait_slow(uint32_t addr, uint32_t parity, int *status,
                                            uint64_t limit, uint32_t fault) {
  volatile AbortRecord *ab = &g_abort;
  uint64_t t0 = global_ns();
  while (!mbar_try_wait_at(addr, parity)) {
    if (ab->set) return;
    if (global_ns() - t0 > limit) {
      flag(status, SQUEEZE_ERR_DEVICE_TIMEOUT);
      ab->bar = addr;
      ab->parity = parity;
      ab->limit = limit;
      ab->status = status;
      ab->nocopy = (fault & SQUEEZE_FAULT_WITHHOLD_LOADS) ? 1u : 0u;
      ab->set = 1u;
      return;
    }
  }
}
__device__ __forceinline__ void mbar_wait(uint64_t *m, uint32_t parity, const TiledDev &p) {
  const uint32_t addr = smem_u32(m);
  if (!mbar_try_wait_at(addr, parity)) mbar_wait_slow(addr, parity, p.status, p.wait_ns, p.fault);
}

// True once a wait of this CTA has given up (read after a CTA barrier, so
// every thread sees the same value).
__device__ __forceinline__ bool cta_aborted() {
  return reinterpret_cast<volatile AbortRecord *>(&g_abort)->set != 0u;
}

// At the end of an aborted launch the copy that timed out may still land in
// shared memory: give it one more bounded wait before the CTA exits.  If it
// still has not landed, it may land in a later CTA's shared memory: the
// status becomes DEVICE_UNSAFE.  (Under the load-withholding hook nothing was
// issued, so there is nothing to wait for.)
__device__ __forceinline__ void settle_abort() {
  if (threadIdx.x == 0 && cta_aborted() && !g_abort.nocopy) {
    const uint64_t t0 = global_ns();
    bool landed = mbar_try_wait_at(g_abort.bar, g_abort.parity);
    while (!landed && global_ns() - t0 < g_abort.limit)
      landed = mbar_try_wait_at(g_abort.bar, g_abort.parity);
    if (!landed) atomicExch(g_abort.status, SQUEEZE_ERR_DEVICE_UNSAFE);
  }
}
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes,
                                          uint64_t *m) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(m))
      : "memory");
}
__device__ __forceinline__ void bulk_store(void *dst, const void *src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(dst),
               "r"(smem_u32(src)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

// Geometry of one group of tiles: band ty, first tile tx0, tile count and the
// byte offset of the group's first row in the compact buffer.
struct Group {
  uint32_t ty, tx0, ntiles, seg;
  uint64_t row0;
};

__device__ __forceinline__ Group group_at(const TiledDev &p, uint32_t TW, uint64_t g) {
  Group G;
  G.ty = fdiv(p.div_gpb, (uint32_t)g);  // groups < 2^32 checked on the host
  G.tx0 = ((uint32_t)g - G.ty * p.groups_per_band) * 32u;
  G.ntiles = min(32u, p.tiles_x - G.tx0);
  G.seg = G.ntiles * TW;
  G.row0 = (uint64_t)G.ty * p.TH * p.W + (uint64_t)G.tx0 * TW;
  return G;
}

// Bytes of row ly that a bulk copy brings in: from the 16-byte aligned start
// A0 up to the segment end rounded up to 16, clipped (to a multiple of 16) at
// the end of the buffer; the few bytes past the clip are loaded by threads.
__device__ __forceinline__ uint32_t row_bulk_bytes(uint64_t S, uint32_t seg, uint64_t total) {
  uint64_t A0 = S & ~(uint64_t)15;
  uint64_t nb = (S - A0 + seg + 15) & ~(uint64_t)15;
  if (A0 + nb > total) nb = (total - A0) & ~(uint64_t)15;
  return (uint32_t)nb;
}

// Warp 0: issue the bulk loads of group G's rows into one staging buffer; the
// buffer's mbarrier completes when all their bytes have landed.
__device__ __forceinline__ void issue_group_loads(const TiledDev &p, const Group &G,
                                                  const uint8_t *in, uint8_t *stage,
                                                  uint64_t *mbar, unsigned lane) {
  const uint64_t W = p.W, total = p.total;
  uint32_t bytes = 0;
  for (uint32_t ly = lane; ly < p.TH; ly += 32)
    bytes += row_bulk_bytes(G.row0 + (uint64_t)ly * W, G.seg, total);
  bytes = __reduce_add_sync(0xFFFFFFFFu, bytes);
  if (lane == 0) mbar_expect_tx(mbar, bytes);
  __syncwarp();
  for (uint32_t ly = lane; ly < p.TH; ly += 32) {
    uint64_t S = G.row0 + (uint64_t)ly * W;
    uint32_t nb = row_bulk_bytes(S, G.seg, total);
    if (nb) bulk_load(stage + (size_t)ly * p.pitch, in + (S & ~(uint64_t)15), nb, mbar);
  }
}

// Rows a warp keeps in flight at once (independent shuffle chains).
constexpr int kRowsInFlight = 3;

// Halo bytes per direction that are loaded ahead of the pack.
constexpr int kHaloAhead = 2;

// Adjacent tile (precomputed table) in direction j of the tile of `lane` in
// group G, or ~0 (a hole or off the box, and for lanes past the group).
__device__ __forceinline__ uint32_t adjacent_of(const TiledDev &p, const Group &G, uint32_t j,
                                                unsigned lane) {
  if (lane >= G.ntiles) return ~0u;
  return __ldg(p.adj + j * p.tiles + (uint64_t)G.ty * p.tiles_x + G.tx0 + lane);
}

// Byte offset of tile t's first cell, or ~0 for t = ~0.
__device__ __forceinline__ uint64_t tile_base(const TiledDev &p, uint32_t TW, uint32_t t) {
  if (t == ~0u) return ~0ull;
  const uint32_t nty = fdiv(p.div_tiles_x, t), ntx = t - nty * p.tiles_x;
  return (uint64_t)nty * p.TH * p.W + (uint64_t)ntx * TW;
}

// Halo words h0 .. h1-1 (one direction): bit `lane` of word h is the state of
// halo reference h of the lane's adjacent tile t (dead for t = ~0).  With
// kBatch > 1 the bytes are loaded kBatch at a time before their ballots, so
// the loads of a direction with many halo cells overlap (the carpet's sides);
// directions with one or two cells (triangle, Vicsek) take the plain loop.
template <int kBatch>
__device__ __forceinline__ void gather_halo(const TiledDev &p, uint32_t TW, uint32_t t,
                                            uint32_t h0, uint32_t h1, const uint32_t *hoff,
                                            uint32_t *words, const uint8_t *in, unsigned lane) {
  const uint64_t base = tile_base(p, TW, t);
  if constexpr (kBatch == 1) {
    for (uint32_t h = h0; h < h1; ++h) {
      bool alive = false;
      if (base != ~0ull) {
        const uint64_t a = base + hoff[h];
        if (a < p.total) alive = __ldg(in + a) & 1u;
        else flag(p.status, SQUEEZE_ERR_DEVICE_BOUNDS);
      }
      const uint32_t word = __ballot_sync(0xFFFFFFFFu, alive);
      if (lane == 0) words[h] = word;
    }
  } else {
  for (uint32_t h = h0; h < h1; h += kBatch) {
    uint32_t v[kBatch];
#pragma unroll
    for (int i = 0; i < kBatch; ++i) {
      v[i] = 0;
      if (h + i < h1 && base != ~0ull) {
        const uint64_t a = base + hoff[h + i];
        if (a < p.total) v[i] = __ldg(in + a);
        else flag(p.status, SQUEEZE_ERR_DEVICE_BOUNDS);
      }
    }
#pragma unroll
    for (int i = 0; i < kBatch; ++i) {
      if (h + i < h1) {
        const uint32_t word = __ballot_sync(0xFFFFFFFFu, v[i] & 1u);
        if (lane == 0) words[h + i] = word;
      }
    }
  }
  }
}

// Halo by chunks (64-wide rows, TiledDev::nchunks > 0).  ctab is the chunk
// table in shared memory: nchunks chunk offsets, nchunks + 1 cell ranges,
// then the cells (halo word | byte << 16).  Lane = tile: each lane loads the
// same 16-byte chunk of its own adjacent tile (base), so one load serves every
// halo cell of that chunk, then each cell's byte becomes one bit of its word.
constexpr int kChunkBatch = 4;   // chunk loads in flight per warp

template <int kB>
__device__ __forceinline__ void load_chunks(const TiledDev &p, uint64_t base,
                                            const uint32_t *ctab, uint32_t c, uint32_t c1,
                                            const uint8_t *in, uint4 *v) {
#pragma unroll
  for (int i = 0; i < kB; ++i) {
    v[i] = make_uint4(0u, 0u, 0u, 0u);
    if (c + i < c1 && base != ~0ull) {
      const uint64_t a = base + ctab[c + i];
      if (a + 16u <= p.total) v[i] = __ldg(reinterpret_cast<const uint4 *>(in + a));
      else flag(p.status, SQUEEZE_ERR_DEVICE_BOUNDS);
    }
  }
}

// Halo words of the cells of chunks c .. min(c + kB, c1) - 1 held in v; cells
// of halo words >= hlimit (rings this launch does not use) are skipped.
template <int kB>
__device__ __forceinline__ void ballot_chunks(const TiledDev &p, const uint32_t *ctab,
                                              uint32_t c, uint32_t c1, const uint4 *v,
                                              uint32_t *words, uint32_t hlimit, unsigned lane) {
  const uint32_t *cstart = ctab + p.nchunks, *cells = cstart + p.nchunks + 1;
#pragma unroll
  for (int i = 0; i < kB; ++i) {
    if (c + i < c1) {
      const uint32_t e1 = cstart[c + i + 1];
      for (uint32_t e = cstart[c + i]; e < e1; ++e) {
        const uint32_t ent = cells[e], h = ent & 0xFFFFu, byte = ent >> 16;
        if (h >= hlimit) break;   // cells are in increasing word order
        const uint32_t w = (byte & 8u) ? ((byte & 4u) ? v[i].w : v[i].z)
                                       : ((byte & 4u) ? v[i].y : v[i].x);
        const uint32_t word = __ballot_sync(0xFFFFFFFFu, (w >> ((byte & 3u) * 8u)) & 1u);
        if (lane == 0) words[h] = word;
      }
    }
  }
}

__device__ __forceinline__ void gather_chunks(const TiledDev &p, uint64_t base,
                                              const uint32_t *ctab, uint32_t c0, uint32_t c1,
                                              uint32_t *words, uint32_t hlimit,
                                              const uint8_t *in, unsigned lane) {
  for (uint32_t c = c0; c < c1; c += kChunkBatch) {
    uint4 v[kChunkBatch];
    load_chunks<kChunkBatch>(p, base, ctab, c, c1, in, v);
    ballot_chunks<kChunkBatch>(p, ctab, c, c1, v, words, hlimit, lane);
  }
}

// Pack tile row ly of the staging buffer into a word (lane = tile; bit 8b + j
// <- byte 4j + b of the row); 0 for lanes past the group.
template <int kTW>
__device__ __forceinline__ uint32_t pack_row(const TiledDev &p, const uint32_t *stage32,
                                             uint32_t o, bool live, uint32_t valid) {
  const uint32_t nwin = kTW ? (3u + (uint32_t)kTW + 3u) / 4u : p.nwin;
  uint32_t acc = 0, acc1 = 0;
  if (live) {
    const uint32_t *w = stage32 + (o >> 2);
    uint32_t sh = (o & 3u) * 8u;
    uint32_t wv[9];
#pragma unroll
    for (int j = 0; j < 9; ++j) wv[j] = (uint32_t)j < nwin ? w[j] : 0u;
#pragma unroll
    for (int j = 0; j < 8; j += 2) {   // two independent chains; the bits do not overlap
      acc |= (__funnelshift_r(wv[j], wv[j + 1], sh) & 0x01010101u) << j;
      acc1 |= (__funnelshift_r(wv[j + 1], wv[j + 2], sh) & 0x01010101u) << (j + 1);
    }
    acc = (acc | acc1) & valid;
  }
  return acc;
}

// Pack a tile row of kTW (8 or 16) bytes that starts on a kTW-byte boundary
// of the staging buffer: kTW / 4 whole words, bit 8b + j <- byte 4j + b.
template <int kTW>
__device__ __forceinline__ uint32_t pack_aligned(const uint32_t *stage32, uint32_t o) {
  uint32_t acc = 0;
  if constexpr (kTW == 8) {
    const uint2 w = *reinterpret_cast<const uint2 *>(stage32 + (o >> 2));
    acc = (w.x & 0x01010101u) | ((w.y & 0x01010101u) << 1);
  } else if constexpr (kTW == 16) {
    const uint4 w = *reinterpret_cast<const uint4 *>(stage32 + (o >> 2));
    acc = (w.x & 0x01010101u) | ((w.y & 0x01010101u) << 1) | ((w.z & 0x01010101u) << 2) |
          ((w.w & 0x01010101u) << 3);
  }
  return acc;
}

// ---- border records -----------------------------------------------------------
//
// rtab: the record table (per record bit: exported cell | halo word << 16, or
// ~0 for padding), read through the cache.  A tile's record word w holds at
// bit i the state of the cell of record bit 32 w + i, so one 32 x 32
// transpose turns the group's words into the 32 tiles' record words and back.

// The records of the group's tiles (bit l of a word = tile l): from the
// exported final words (words[e], map null) or from the word array of the
// group (words[map[e]], map = the exported cells' slots).  Warp-strided over
// record words; lane l stores its tile's.
__device__ __forceinline__ void build_records(const TiledDev &p, const uint32_t *words,
                                              const uint32_t *map, const Group &G,
                                              const uint32_t *rtab, uint32_t *rec_out,
                                              unsigned lane, unsigned warp, unsigned nw,
                                              const uint32_t *keep, const uint32_t *rot) {
  const uint32_t R = p.rec_words;
  const uint64_t t0 = (uint64_t)G.ty * p.tiles_x + G.tx0;
  for (uint32_t w = warp; w < R; w += nw) {
    const uint32_t e = __ldg(rtab + 32u * w + lane);
    uint32_t x = 0u;
    if (e != 0xFFFFFFFFu) x = words[map ? __ldg(map + (e & 0xFFFFu)) : (e & 0xFFFFu)];
    transpose32_n<1>(&x, keep, rot);
    if (lane < G.ntiles) rec_out[(t0 + lane) * R + w] = x;
  }
}

// Halo words of direction j from the records of the lanes' adjacent tiles t
// (~0: none, all dead): lane l loads record word w of its tile, and after the
// transpose lane i holds the word of record bit 32 w + i, whose halo word the
// table names.  Words of rings past hlimit are skipped.
template <int kN>
__device__ __forceinline__ void records_to_words(const TiledDev &p, uint32_t t, uint32_t w,
                                                 const uint32_t *rtab, const uint32_t *rec_in,
                                                 uint32_t *words, uint32_t hlimit, unsigned lane,
                                                 const uint32_t *keep, const uint32_t *rot) {
  uint32_t x[kN];
#pragma unroll
  for (int i = 0; i < kN; ++i)
    x[i] = t != ~0u ? __ldg(rec_in + (uint64_t)t * p.rec_words + w + i) : 0u;
  transpose32_n<kN>(x, keep, rot);
#pragma unroll
  for (int i = 0; i < kN; ++i) {
    const uint32_t e = __ldg(rtab + 32u * (w + i) + lane), h = e >> 16;
    if (e != 0xFFFFFFFFu && h < hlimit) words[h] = x[i];
  }
}

__device__ __forceinline__ void gather_records(const TiledDev &p, uint32_t t, uint32_t j,
                                               const uint32_t *rtab, const uint32_t *rec_in,
                                               uint32_t *words, uint32_t hlimit, unsigned lane,
                                               const uint32_t *keep, const uint32_t *rot) {
  const uint32_t w1 = p.rec_seg[j + 1];
  if (t != ~0u && t >= p.tiles) {
    flag(p.status, SQUEEZE_ERR_DEVICE_BOUNDS);
    t = ~0u;
  }
  uint32_t w = p.rec_seg[j];
  for (; w + 2u <= w1; w += 2u)   // two words per transpose pass
    records_to_words<2>(p, t, w, rtab, rec_in, words, hlimit, lane, keep, rot);
  if (w < w1) records_to_words<1>(p, t, w, rtab, rec_in, words, hlimit, lane, keep, rot);
}

// Pack a 64-byte tile row at o (16-byte aligned; lane = tile, the lanes' rows
// 64 bytes apart) into two words, one per 32-byte half: bit 8b + j of a half's
// word <- byte 4j + b of the half.  Lane l reads the row's four 16-byte chunks
// starting at chunk rot = (l >> 1) & 3, so the 8 lanes of each phase of a
// 16-byte shared load touch 8 different bank groups (reading chunk c in every
// lane would put lanes l, l + 2, l + 4, l + 6 on the same banks).
__device__ __forceinline__ void pack_row64(const uint32_t *stage32, uint32_t o, uint32_t rot,
                                           uint32_t &lo, uint32_t &hi) {
  uint32_t a0 = 0, a1 = 0;
#pragma unroll
  for (uint32_t c = 0; c < 4; ++c) {
    const uint32_t q = (c + rot) & 3u;   // chunk of the row read at this step
    const uint4 v = *reinterpret_cast<const uint4 *>(stage32 + (o >> 2) + q * 4u);
    const uint32_t j = (q & 1u) * 4u;    // its first word within its half
    const uint32_t m = ((v.x & 0x01010101u) << j) | ((v.y & 0x01010101u) << (j + 1u)) |
                       ((v.z & 0x01010101u) << (j + 2u)) | ((v.w & 0x01010101u) << (j + 3u));
    a0 |= (q >> 1) ? 0u : m;
    a1 |= (q >> 1) ? m : 0u;
  }
  lo = a0;
  hi = a1;
}

// The inverse of pack_row64, with the same chunk rotation.
__device__ __forceinline__ void unpack_row64(uint32_t *stage32w, uint32_t o, uint32_t rot,
                                             uint32_t lo, uint32_t hi) {
#pragma unroll
  for (uint32_t c = 0; c < 4; ++c) {
    const uint32_t q = (c + rot) & 3u;
    const uint32_t y = (q >> 1) ? hi : lo, j = (q & 1u) * 4u;
    *reinterpret_cast<uint4 *>(stage32w + (o >> 2) + q * 4u) =
        make_uint4((y >> j) & 0x01010101u, (y >> (j + 1u)) & 0x01010101u,
                   (y >> (j + 2u)) & 0x01010101u, (y >> (j + 3u)) & 0x01010101u);
  }
}

// The inverse of pack_aligned: the low kTW / 4 bit planes of y, as whole words.
template <int kTW>
__device__ __forceinline__ void unpack_aligned(uint32_t *stage32w, uint32_t o, uint32_t y) {
  if constexpr (kTW == 8) {
    *reinterpret_cast<uint2 *>(stage32w + (o >> 2)) =
        make_uint2(y & 0x01010101u, (y >> 1) & 0x01010101u);
  } else if constexpr (kTW == 16) {
    *reinterpret_cast<uint4 *>(stage32w + (o >> 2)) =
        make_uint4(y & 0x01010101u, (y >> 1) & 0x01010101u, (y >> 2) & 0x01010101u,
                   (y >> 3) & 0x01010101u);
  }
}

// Unpack a packed row word y into bytes and write them at staging offset o;
// a word shared with the neighbouring lane's segment is handed to the
// right-hand lane, which merges it.
template <int kTW>
__device__ __forceinline__ void unpack_row(uint32_t *stage32w, uint8_t *stage, uint32_t y,
                                           uint32_t o, uint32_t TW, unsigned lane,
                                           uint32_t ntiles) {
  if (TW >= 4) {
    uint32_t shb = o & 3u, sh = shb * 8u, base = o >> 2;
    uint32_t u[9], prev = 0;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      uint32_t v = (y >> t) & 0x01010101u;
      u[t] = __funnelshift_l(prev, v, sh);
      prev = v;
    }
    u[8] = __funnelshift_l(prev, 0u, sh);
    uint32_t E = (shb + TW - 1) >> 2;
    bool partial = ((shb + TW) & 3u) != 0;
    uint32_t last;
    if constexpr (kTW != 0) {
      constexpr uint32_t E0 = kTW > 0 ? ((uint32_t)kTW - 1u) >> 2 : 0u;
      last = E == E0 ? u[E0] : u[E0 + 1 < 9 ? E0 + 1 : 8];
    } else {
      last = 0;
#pragma unroll
      for (int t = 0; t < 9; ++t) last = (uint32_t)t == E ? u[t] : last;
    }
    uint32_t recv = __shfl_up_sync(0xFFFFFFFFu, partial ? last : 0u, 1);
    if (lane >= 1) u[0] |= recv;
    bool give = partial && lane + 1 < ntiles;
    if (lane < ntiles) {
      if constexpr (kTW != 0) {
        constexpr uint32_t E0 = kTW > 0 ? ((uint32_t)kTW - 1u) >> 2 : 0u;
#pragma unroll
        for (uint32_t t = 0; t < E0; ++t) stage32w[base + t] = u[t];
        if (E > E0 || !give) stage32w[base + E0] = u[E0];
        if (E0 + 1 < 9 && E > E0 && !give) stage32w[base + E0 + 1] = u[E0 + 1 < 9 ? E0 + 1 : 8];
      } else {
#pragma unroll
        for (int t = 0; t < 9; ++t)
          if ((uint32_t)t < E || ((uint32_t)t == E && !give)) stage32w[base + t] = u[t];
      }
    }
  } else if (lane < ntiles) {
    for (uint32_t bb = 0; bb < TW; ++bb) {
      uint32_t L = 8u * (bb & 3u) + (bb >> 2);
      stage[o + bb] = (uint8_t)((y >> L) & 1u);
    }
  }
}

// Shared-memory carve-up of the tiled kernel (offsets in bytes; every region
// starts at a multiple of 16): two word buffers, halo offsets, halo
// directions, 2 mbarriers, two sets of row offsets, the row-end carry chunks,
// the final-step words of two groups (border records only), two staging
// buffers.
struct SmemPtrs {
  unsigned char *win0;
  uint32_t *hoff;
  uint8_t *hdir;
  uint64_t *mbar;
  uint8_t *rowa;
  uint8_t *carry;
  uint32_t *z;      // final-step words of the last two groups (border records)
  uint8_t *stage0;
};

__device__ __forceinline__ SmemPtrs carve(unsigned char *smem, const TileLayout &lay) {
  SmemPtrs q;
  size_t off = 0;
  q.win0 = smem;
  off += 2 * (size_t)lay.win_bytes;
  q.hoff = reinterpret_cast<uint32_t *>(smem + off);
  off += lay.hoff_bytes;
  q.hdir = smem + off;
  off += lay.hdir_bytes;
  q.mbar = reinterpret_cast<uint64_t *>(smem + off);
  off += 16;
  q.rowa = smem + off;
  off += lay.rowa_bytes;
  q.carry = smem + off;
  off += lay.carry_bytes;
  q.z = reinterpret_cast<uint32_t *>(smem + off);
  off += lay.z_bytes;
  q.stage0 = smem + off;
  return q;
}

// The rule applied to word c of a word array: its 8 neighbour words by the
// program's byte offsets (one 16-byte table load), the word itself as "alive".
template <bool kLife>
__device__ __forceinline__ uint32_t rule_at(const TiledDev &p, const unsigned char *wbase,
                                            uint32_t c) {
  const uint4 r4 = __ldg(reinterpret_cast<const uint4 *>(p.refs) + c);
  const uint32_t rw[4] = {r4.x, r4.y, r4.z, r4.w};
  uint32_t n[8];
#pragma unroll
  for (int d = 0; d < 4; ++d) {
    n[2 * d] = *reinterpret_cast<const uint32_t *>(wbase + __byte_perm(rw[d], 0, 0x4410));
    n[2 * d + 1] = *reinterpret_cast<const uint32_t *>(wbase + __byte_perm(rw[d], 0, 0x4432));
  }
  return rule_word<kLife>(p.rule, reinterpret_cast<const uint32_t *>(wbase)[c], n);
}

// One pass of the tiled step over groups g_first, g_first + g_stride, ...
// (< g_end) of one fractal instance, by one CTA.
//
// The caller is instantiated for the common tile-row widths so that the word
// counts of a row are compile-time constants; kTW = 0 takes TW at run time.
//
// Work split inside the CTA: warp w owns units u = w, w + nw, ... of every
// group (a unit is a slot row, i.e. one tile row or the rows sharing one
// word, or for 64-wide rows one tile row of two slot rows), from packing
// through the rule to the write-back, and keeps several slot rows in flight.
// The word array is double-buffered by
// group, so one CTA barrier per group suffices (before the rule reads the
// words): a warp that passed it knows every warp finished the group before,
// whose word buffer and staging buffer may then be reused.  Warp w also
// resolves directions j = w, w + nw, ... of the tiles' adjacent tiles and
// gathers their halo words.  While group i is processed in staging buffer
// i % 2, the bulk loads of group i + 1 land in the other one.  `it` counts
// the groups this CTA has processed (it selects buffers and mbarrier phases)
// and carries over from one call to the next.
//
// kT = 2, 4 or 8 (steps per launch): the packed words of a group go to word
// buffer X (buffer 0), together with halo rings 1..kT and the per-direction
// masks of which adjacent tiles exist.  After the barrier, rule pass t
// (t = 1 .. kT - 1) writes step t of every slot and of rings 1..kT-t from one
// buffer into the other (X -> Y, Y -> X, X -> Y; a ring cell of a missing
// tile stays dead), each followed by a barrier, and the final rule pass
// computes step kT from Y and writes it back.  X's last reader is pass kT - 1
// and Y's the final pass, so the next group can fill X after the final pass
// and Y after its own first barrier: two buffers suffice for an even kT.
template <bool kLife, int kTW, int kT>
__device__ __forceinline__ void run_groups(const TiledDev &p, const TileLayout &lay,
                                           const uint8_t *__restrict__ in,
                                           uint8_t *__restrict__ out, uint64_t g_first,
                                           uint64_t g_end, uint64_t g_stride,
                                           unsigned char *smem, const uint32_t *keep,
                                           const uint32_t *rot, uint32_t &it,
                                           const uint32_t *rec_in, uint32_t *rec_out,
                                           bool rec_only) {
  // Tile rows per slot word (kTW = 8, 16: the rows of 4 or 2 tile rows share
  // one word), slot rows in flight per warp, and tile rows per write-back batch.
  // (kTW = 64: each tile row is two slot words, its left and right halves; a
  // warp keeps both halves of its rows.)  Units are what a warp owns: slot
  // rows (kWPR = 1) or tile rows (kWPR = 2).
  constexpr uint32_t kRPW = kTW == 8 ? 4u : (kTW == 16 ? 2u : 1u);
  constexpr uint32_t kWPR = kTW == 64 ? 2u : 1u;
  constexpr int kR = kRPW > 1 ? 2 : (kWPR > 1 ? 4 : kRowsInFlight);
  constexpr uint32_t kRR = kRPW > 1 ? (uint32_t)kR * kRPW : (uint32_t)kR / kWPR;
  constexpr uint32_t kU = (uint32_t)kR / kWPR;   // units per pass
  constexpr int kHaloBatch = kTW == 27 || kTW == 25 ? 1 : 4;
  const uint32_t slots = p.slots, nhalo = p.nhalo;
  const uint32_t TW = kTW ? (uint32_t)kTW : p.TW;
  const uint32_t VR = p.TH * kWPR / kRPW;   // slot rows
  const uint32_t NU = VR / kWPR;            // units
  const SmemPtrs q = carve(smem, lay);
  const size_t win_bytes = lay.win_bytes, stage_bytes = lay.stage_bytes;
  uint32_t *hoff = q.hoff;
  uint8_t *hdir = q.hdir;
  uint64_t *mbar = q.mbar;
  uint8_t *rowa = q.rowa;
  uint8_t *carry = q.carry;
  uint8_t *stage_base = q.stage0;

  const unsigned tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
  const unsigned nthreads = blockDim.x, nw = nthreads >> 5;
  // Slot row of entry k of the pass that starts at unit u0.
  auto vrow = [&](uint32_t u0, int k) -> uint32_t {
    return kWPR * (u0 + ((uint32_t)k / kWPR) * nw) + (uint32_t)k % kWPR;
  };
  __syncthreads();  // the previous call (another instance) is done with every buffer
  // A CTA that gave up on an earlier instance of a batch loads nothing more:
  // this instance's output is not valid either, so its status says so.
  if (tid == 0 && cta_aborted()) flag(p.status, SQUEEZE_ERR_DEVICE_TIMEOUT);
  // 64-wide rows gather the halo by chunks (their programs always carry the
  // chunk table); the table follows the halo offsets in global and in shared
  // memory.
  constexpr bool kChunked = kTW == 64;
  const uint32_t ntab = nhalo + (kChunked && p.nchunks ? 2u * p.nchunks + 1u + nhalo : 0u);
  const uint32_t *ctab = hoff + nhalo;
  // Border records (programs with a record table): read the input's records
  // for the halo (rec_in; else gather from the state), write the output's
  // (rec_out); rec_only: write the input's records to rec_out and nothing else.
  // The record tables stay in device memory (read through the cache): record
  // bits (exported cell | halo word << 16), the exported cells' slots, and
  // each slot's exported cell (16 bits).
  const uint32_t *rtab = p.halo_off + ntab;
  const uint32_t *exp_slot = rtab + 32u * p.rec_words;
  const uint16_t *exp_of = reinterpret_cast<const uint16_t *>(exp_slot + p.rec_nexp);
  const bool use_rec = p.rec_words != 0u && rec_in != nullptr;
  const bool produce = p.rec_words != 0u && rec_out != nullptr && !rec_only;
  // Halo gathered after the pack (records, or chunks of 64-wide rows), or
  // byte by byte.  Launches of more than one step always have the input's
  // records, so only one-step launches (the allocation-free step has no
  // records) compile the gathers from the state.
  constexpr bool kGather = kT == 1;
  const bool deferred = !kGather || kChunked || use_rec || rec_only;
  const uint32_t nexp = p.rec_nexp;
  uint32_t *zbuf = q.z;   // exported final words of the last two groups
  for (uint32_t i = tid; i < ntab; i += nthreads) hoff[i] = p.halo_off[i];
  if constexpr (kT > 1)
    for (uint32_t i = tid; i < p.ring_end[kT - 1]; i += nthreads) hdir[i] = p.halo_dir[i];
  if (tid == 0) {
    reinterpret_cast<uint32_t *>(smem)[slots + nhalo] = 0u;  // "no neighbour" words
    reinterpret_cast<uint32_t *>(smem + win_bytes)[slots + nhalo] = 0u;
  }
  __syncthreads();  // halo offsets and zero words in place
  const uint64_t total = p.total, W = p.W;
  const uint32_t valid = p.valid;

  const bool withhold = (p.fault & SQUEEZE_FAULT_WITHHOLD_LOADS) != 0u;  // test hook
  if (warp == 0 && g_first < g_end && !cta_aborted() && !withhold)
    issue_group_loads(p, group_at(p, TW, g_first), in, stage_base + (it & 1u) * stage_bytes,
                      &mbar[it & 1u], lane);
  // Adjacent tile of this lane's tile in direction j = warp, for the group at hand.
  uint32_t t_cur = ~0u;
  if (warp < p.ndirs && g_first < g_end)
    t_cur = adjacent_of(p, group_at(p, TW, g_first), warp, lane);

  for (uint64_t g = g_first; g < g_end; g += g_stride, ++it) {
    const uint32_t b = it & 1u;
    // Word buffer of the packed input: by group parity for one step per
    // launch; buffer 0 (X) for more.
    unsigned char *wbase = smem + (kT > 1 ? 0u : b) * win_bytes;
    uint32_t *win = reinterpret_cast<uint32_t *>(wbase);
    uint32_t *emask = win + slots + nhalo + 1;   // kT > 1: which adjacent tiles exist, per direction
    uint8_t *stage = stage_base + b * stage_bytes;
    const uint32_t *stage32 = reinterpret_cast<const uint32_t *>(stage);
    uint32_t *stage32w = reinterpret_cast<uint32_t *>(stage);
    const Group G = group_at(p, TW, g);
    const uint32_t ntiles = G.ntiles, seg = G.seg;
    // A row segment shares its first and last 16-byte chunk with the groups
    // beside it.  When the next group of the band is also this CTA's next
    // group, the last partial chunk of each row is handed to it in `carry`
    // (row ly stays with the same warp from group to group) instead of being
    // written in pieces, and that group completes the chunk with its own
    // first bytes and stores it whole.
    const bool has_prev = g_stride == 1 && g > g_first && G.tx0 != 0;
    const bool gives = g_stride == 1 && g + 1 < g_end && G.tx0 + 32u < p.tiles_x;

    // This warp's bulk stores of the previous group must finish reading the
    // other staging buffer before the CTA barrier below lets it be refilled.
    bulk_wait_read();

    // Halo words, one direction per warp.  Direction j = warp (the common
    // case): its adjacent tiles were looked up during the previous group;
    // the first kHaloAhead halo bytes are loaded now and turned into words
    // after the pack below, so their latency overlaps the pack.  The rest,
    // and directions j >= nw, are gathered in place.
    uint32_t hb[kHaloAhead];
    uint32_t h_pre = 0, t_next = ~0u;
    const uint32_t hlimit = p.ring_end[kT];   // halo words of the rings this launch uses
    if (deferred && warp < p.ndirs) {
      // chunks or records: direction `warp` is gathered after the pack (loading
      // chunks ahead of it costs registers and measured no faster)
      if (g + g_stride < g_end) t_next = adjacent_of(p, group_at(p, TW, g + g_stride), warp, lane);
      if constexpr (kT > 1) {
        const uint32_t m = __ballot_sync(0xFFFFFFFFu, t_cur != ~0u);
        if (lane == 0) emask[warp] = m;
      }
    } else if (kGather && !deferred && warp < p.ndirs) {
      const uint32_t h0 = p.halo_start[warp], h1 = p.halo_start[warp + 1];
      h_pre = min(h1 - h0, (uint32_t)kHaloAhead);
      const uint64_t base = tile_base(p, TW, t_cur);
#pragma unroll
      for (int i = 0; i < kHaloAhead; ++i) {
        hb[i] = 0;
        if ((uint32_t)i < h_pre && base != ~0ull) {
          const uint64_t a = base + hoff[h0 + i];
          if (a < total) hb[i] = __ldg(in + a);
          else flag(p.status, SQUEEZE_ERR_DEVICE_BOUNDS);
        }
      }
      if (g + g_stride < g_end) t_next = adjacent_of(p, group_at(p, TW, g + g_stride), warp, lane);
      if constexpr (kT > 1) {
#pragma unroll
        for (int k = 0; k < kT - 1; ++k)   // rings 2 .. kT
          gather_halo<kHaloBatch>(p, TW, t_cur, p.ring_start[k][warp], p.ring_start[k][warp + 1],
                                  hoff, win + slots, in, lane);
        const uint32_t m = __ballot_sync(0xFFFFFFFFu, t_cur != ~0u);
        if (lane == 0) emask[warp] = m;
      }
    }
    for (uint32_t j = warp + nw; j < p.ndirs; j += nw) {
      const uint32_t t = adjacent_of(p, G, j, lane);
      if (deferred) {
        if (rec_only) {
        } else if (use_rec) {
          gather_records(p, t, j, rtab, rec_in, win + slots, hlimit, lane, keep, rot);
        } else if constexpr (kChunked && kGather) {
          gather_chunks(p, tile_base(p, TW, t), ctab, p.chunk_start[j], p.chunk_start[j + 1],
                        win + slots, hlimit, in, lane);
        }
      } else if constexpr (kGather) {
        gather_halo<kHaloBatch>(p, TW, t, p.halo_start[j], p.halo_start[j + 1], hoff,
                                win + slots, in, lane);
        if constexpr (kT > 1) {
#pragma unroll
          for (int k = 0; k < kT - 1; ++k)
            gather_halo<kHaloBatch>(p, TW, t, p.ring_start[k][j], p.ring_start[k][j + 1], hoff,
                                    win + slots, in, lane);
        }
      }
      if constexpr (kT > 1) {
        const uint32_t m = __ballot_sync(0xFFFFFFFFu, t != ~0u);
        if (lane == 0) emask[j] = m;
      }
    }

    mbar_wait(&mbar[b], (it >> 1) & 1u, p);
    // Bytes past the last 16-byte boundary of the buffer (only rows that end
    // within 16 bytes of it) were not part of a bulk copy: load them here.
    if (G.row0 + (uint64_t)(p.TH - 1) * W + seg + 16 > total) {
      for (uint32_t ly = warp; ly < p.TH; ly += nw) {
        const uint64_t S = G.row0 + (uint64_t)ly * W, A0 = S & ~(uint64_t)15;
        const uint64_t got = A0 + row_bulk_bytes(S, seg, total);
        for (uint64_t a = got + lane; a < S + seg; a += 32)
          stage[(size_t)ly * p.pitch + (uint32_t)(a - A0)] = in[a];
      }
      __syncwarp();
    }

    // Pack the own tile rows into words (lane = tile) and transpose them so
    // that lane L holds local cell (ly, lx(L)) of all 32 tiles.
    for (uint32_t u0 = warp; u0 < NU; u0 += kU * nw) {
      uint32_t acc[kR];
#pragma unroll
      for (int k = 0; k < kR; ++k) {
        const uint32_t vr = vrow(u0, k);
        if constexpr (kWPR > 1) {
          // entries k, k + 1 are the two halves of one tile row (a row starts on
          // a 64-byte boundary: its alignment offset a is 0)
          if (k % 2 == 0) {
            acc[k] = acc[k + 1] = 0;
            if (vr < VR) {
              const uint32_t ly = vr / kWPR, a = ((uint32_t)G.row0 + ly * (uint32_t)W) & 15u;
              if (lane == 0) rowa[b * p.TH + ly] = (uint8_t)a;
              if (lane < ntiles)
                pack_row64(stage32, ly * p.pitch + a + lane * 64u, (lane >> 1) & 3u, acc[k],
                           acc[k + 1]);
            }
          }
        } else if constexpr (kRPW == 1) {
          const uint32_t ly = vr;
          const uint32_t a = ((uint32_t)G.row0 + ly * (uint32_t)W) & 15u;
          if (lane == 0 && ly < p.TH) rowa[b * p.TH + ly] = (uint8_t)a;
          acc[k] = pack_row<kTW>(p, stage32, ly * p.pitch + a + lane * TW,
                                 ly < p.TH && lane < ntiles, valid);
        } else {
          acc[k] = 0;
          if (vr < VR) {
#pragma unroll
            for (uint32_t i = 0; i < kRPW; ++i) {
              const uint32_t ly = vr * kRPW + i;
              const uint32_t a = ((uint32_t)G.row0 + ly * (uint32_t)W) & 15u;
              if (lane == 0) rowa[b * p.TH + ly] = (uint8_t)a;
              if (lane < ntiles)
                acc[k] |= pack_aligned<kTW>(stage32, ly * p.pitch + a + lane * (uint32_t)kTW)
                          << (i * (uint32_t)(kTW / 4));
            }
          }
        }
      }
      transpose32_n<kR>(acc, keep, rot);
#pragma unroll
      for (int k = 0; k < kR; ++k)
        if (vrow(u0, k) < VR) win[vrow(u0, k) * 32u + lane] = acc[k];
    }
    if (deferred && warp < p.ndirs) {
      if (rec_only) {
      } else if (use_rec) {
        gather_records(p, t_cur, warp, rtab, rec_in, win + slots, hlimit, lane, keep, rot);
      } else if constexpr (kChunked && kGather) {
        gather_chunks(p, tile_base(p, TW, t_cur), ctab, p.chunk_start[warp],
                      p.chunk_start[warp + 1], win + slots, hlimit, in, lane);
      }
      t_cur = t_next;
    } else if (kGather && !deferred && warp < p.ndirs) {
      const uint32_t h0 = p.halo_start[warp];
#pragma unroll
      for (int i = 0; i < kHaloAhead; ++i) {
        if ((uint32_t)i < h_pre) {
          const uint32_t word = __ballot_sync(0xFFFFFFFFu, hb[i] & 1u);
          if (lane == 0) win[slots + h0 + i] = word;
        }
      }
      if (h0 + h_pre < p.halo_start[warp + 1])
        gather_halo<kHaloBatch>(p, TW, t_cur, h0 + h_pre, p.halo_start[warp + 1], hoff, win + slots,
                                in, lane);
      t_cur = t_next;
    }
    // The only CTA barrier of the group: all words (rows and halo) are in
    // place, and every warp has finished the previous group.
    __syncthreads();
    if (warp == 0 && g + g_stride < g_end && !cta_aborted() && !withhold)
      issue_group_loads(p, group_at(p, TW, g + g_stride), in, stage_base + (b ^ 1u) * stage_bytes,
                        &mbar[b ^ 1u], lane);
    if (rec_only) {   // the input's records from its packed words; no step
      build_records(p, win, exp_slot, G, rtab, rec_out, lane, warp, nw, keep, rot);
      continue;
    }
    // The previous group's records: its exported final words are complete,
    // since every warp has passed this barrier (and nothing rewrites them
    // before the next one).
    if (produce && g != g_first)
      build_records(p, zbuf + ((it - 1u) & 1u) * nexp, nullptr, group_at(p, TW, g - g_stride),
                    rtab, rec_out, lane, warp, nw, keep, rot);

    // kT > 1: steps 1 .. kT-1 of the own slot rows and of the halo rings that
    // the later steps still need, alternating between X and Y.
    const unsigned char *rbase = wbase;   // the words the final rule pass reads
    if constexpr (kT > 1) {
#pragma unroll 1
      for (int t = 1; t < kT; ++t) {
        const unsigned char *src = smem + (t & 1 ? 0u : win_bytes);
        uint32_t *dst = reinterpret_cast<uint32_t *>(smem + (t & 1 ? win_bytes : 0u));
        for (uint32_t u0 = warp; u0 < NU; u0 += kU * nw) {
          uint32_t nx[kR];
#pragma unroll
          for (int k = 0; k < kR; ++k)
            nx[k] = vrow(u0, k) < VR ? rule_at<kLife>(p, src, vrow(u0, k) * 32u + lane) : 0u;
#pragma unroll
          for (int k = 0; k < kR; ++k)
            if (vrow(u0, k) < VR) dst[vrow(u0, k) * 32u + lane] = nx[k];
        }
        // (rings from the last warp down: warp 0 issues the loads and the low
        // warps gather halo bytes, so the last warps have the least other work)
        for (uint32_t i = (nw - 1u - warp) * 32u + lane; i < p.ring_end[kT - t]; i += nw * 32u)
          dst[slots + i] = rule_at<kLife>(p, src, slots + i) & emask[hdir[i]];
        __syncthreads();   // step t complete; every warp is done reading src
      }
      rbase = smem + win_bytes;   // Y: kT is even
    }

    // Rule, inverse transpose and write-back of the own rows.
    for (uint32_t u0 = warp; u0 < NU; u0 += kU * nw) {
      uint32_t y[kR];
#pragma unroll
      for (int k = 0; k < kR; ++k)
        y[k] = vrow(u0, k) < VR ? rule_at<kLife>(p, rbase, vrow(u0, k) * 32u + lane) : 0u;
      if (produce) {   // keep the exported final words for this group's records
#pragma unroll
        for (int k = 0; k < kR; ++k)
          if (vrow(u0, k) < VR) {
            const uint32_t e = __ldg(exp_of + vrow(u0, k) * 32u + lane);
            if (e != 0xFFFFu) zbuf[(it & 1u) * nexp + e] = y[k];
          }
      }
      transpose32_n<kR>(y, keep, rot);
      // Row offsets first: a shared load after the unpack's stores would wait for them.
      uint32_t arow[kR];
#pragma unroll
      for (int k = 0; k < kR; ++k) {
        const uint32_t ly = kWPR > 1 ? vrow(u0, k) / kWPR : vrow(u0, k);
        arow[k] = kRPW == 1 && vrow(u0, k) < VR ? rowa[b * p.TH + ly] : 0u;
      }
#pragma unroll
      for (int k = 0; k < kR; ++k) {
        const uint32_t vr = vrow(u0, k);
        if constexpr (kWPR > 1) {
          if (k % 2 == 0 && vr < VR && lane < ntiles)
            unpack_row64(stage32w, vr / kWPR * p.pitch + arow[k] + lane * 64u, (lane >> 1) & 3u,
                         y[k], y[k + 1]);
        } else if constexpr (kRPW == 1) {
          const uint32_t ly = vr;
          if (ly < p.TH)
            unpack_row<kTW>(stage32w, stage, y[k] & valid, ly * p.pitch + arow[k] + lane * TW, TW,
                            lane, ntiles);
        } else if (vr < VR && lane < ntiles) {
#pragma unroll
          for (uint32_t i = 0; i < kRPW; ++i) {
            const uint32_t ly = vr * kRPW + i;
            unpack_aligned<kTW>(stage32w, ly * p.pitch + rowa[b * p.TH + ly] + lane * (uint32_t)kTW,
                                y[k] >> (i * (uint32_t)(kTW / 4)));
          }
        }
      }
      __syncwarp();
      // Tile row of entry rr of this write-back batch (rr < kRR); >= TH past the end.
      auto row_of = [&](uint32_t rr) -> uint32_t {
        if constexpr (kRPW > 1) {
          const uint32_t vr = u0 + (rr / kRPW) * nw;
          return vr < VR ? vr * kRPW + rr % kRPW : p.TH;
        } else {
          return u0 + rr * nw;   // a unit is a tile row (>= TH past the end)
        }
      };
      // Carried chunks: take the previous group's tail bytes in front of the
      // row (staging offsets [0, a)), hand this row's tail on.
      if (has_prev || gives) {
        for (uint32_t e = lane; e < 16u * kRR; e += 32u) {
          const uint32_t i = e & 15u, ly = row_of(e >> 4);
          if (ly < p.TH) {
            const uint32_t a = rowa[b * p.TH + ly], end = a + seg;
            uint8_t *sb = stage + ly * p.pitch;
            if (has_prev && i < a) sb[i] = carry[ly * 16u + i];
            if (gives && i < (end & 15u)) carry[ly * 16u + i] = sb[(end & ~15u) + i];
          }
        }
      }
      // Write the rows.  In staging offsets (offset 0 is the 16-byte aligned
      // address below the row start) the bytes [v0, v1) go out: one bulk store
      // per row for the whole chunks [m0, m1) (lane k issues row k) and, for
      // each ragged end (a chunk shared with a neighbouring group), up to four
      // aligned pieces of 8/4/2/1 bytes (lane 2k + side).
      fence_async_smem();
      __syncwarp();
      // (With a carried chunk at both ends no row has an edge piece.)
      if (lane < (has_prev && gives ? 1u : 3u) * kRR) {  // [0, RR): bulk; [RR, 3RR): edges
        const uint32_t ly = row_of(lane < kRR ? lane : (lane - kRR) >> 1);
        if (ly < p.TH) {
          const uint32_t a = rowa[b * p.TH + ly], end = a + seg;
          const uint32_t v0 = has_prev ? 0u : a, v1 = gives ? (end & ~15u) : end;
          const uint32_t m0 = (v0 + 15u) & ~15u, m1 = v1 & ~15u;
          const bool split = m0 < m1;
          uint8_t *g0 = out + (G.row0 + (uint64_t)ly * W - a);  // staging offset 0 in HBM
          const uint8_t *s0 = stage + ly * p.pitch;
          if (lane < kRR) {
            if (split) bulk_store(g0 + m0, s0 + m0, m1 - m0);
          } else {
            // side 0: [v0, m0) or all of [v0, v1) when there is no middle;
            // side 1: [m1, v1).
            const bool side = (lane - kRR) & 1u;
            uint32_t lo = side ? m1 : v0, hi = side ? v1 : (split ? m0 : v1);
            if (side && !split) hi = lo = 0;
            while (lo < hi) {
              const uint32_t n = hi - lo, al = lo;
              if ((al & 1u) || n < 2) { g0[lo] = s0[lo]; lo += 1; }
              else if ((al & 2u) || n < 4) {
                *reinterpret_cast<uint16_t *>(g0 + lo) = *reinterpret_cast<const uint16_t *>(s0 + lo);
                lo += 2;
              } else if ((al & 4u) || n < 8) {
                *reinterpret_cast<uint32_t *>(g0 + lo) = *reinterpret_cast<const uint32_t *>(s0 + lo);
                lo += 4;
              } else {
                *reinterpret_cast<uint2 *>(g0 + lo) = *reinterpret_cast<const uint2 *>(s0 + lo);
                lo += 8;
              }
            }
          }
        }
      }
      if (lane < kRR) bulk_commit();
    }
  }
  // the last group's records (after a barrier: its final words are complete)
  if (produce && g_first < g_end) {
    __syncthreads();
    const uint64_t last = g_first + (g_end - 1u - g_first) / g_stride * g_stride;
    build_records(p, zbuf + ((it - 1u) & 1u) * nexp, nullptr, group_at(p, TW, last), rtab,
                  rec_out, lane, warp, nw, keep, rot);
  }
}


// Mbarriers of the two staging buffers, set up once per CTA.
__device__ __forceinline__ void init_barriers(unsigned char *smem, const TileLayout &lay) {
  if (threadIdx.x == 0) {
    uint64_t *mbar = carve(smem, lay).mbar;
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    g_abort.set = 0u;
  }
}

// kT steps (1, 2, 4 or 8) of one instance; CTA c of the persistent grid takes
// the contiguous run of groups [c G / grid, (c + 1) G / grid), except for
// 64-wide rows: there CTA c takes groups c, c + grid, c + 2 grid, ..., so that
// the CTAs work on a band of neighbouring groups at a time and the halo chunks
// they read from the tiles above and below are still in L2 (those rows start
// on 16-byte boundaries, so nothing is lost by not handing row ends over).
template <bool kLife, int kTW, int kT>
__global__ void __launch_bounds__(kTW == 64 ? 256 : kTiledMaxThreads) step_tiled_kernel(
    TiledDev p, TileLayout lay, const uint8_t *__restrict__ in, uint8_t *__restrict__ out) {
  extern __shared__ __align__(128) unsigned char smem[];
  uint32_t keep[5], rot[5];
  make_transpose(threadIdx.x & 31u, keep, rot);
  init_barriers(smem, lay);
  uint32_t it = 0;
  if constexpr (kTW == 64) {
    run_groups<kLife, kTW, kT>(p, lay, in, out, blockIdx.x, p.groups, gridDim.x, smem, keep, rot,
                               it, p.rec[0], p.rec[1], p.mode == 1u);
  } else {
    const uint64_t g0 = (uint64_t)blockIdx.x * p.groups / gridDim.x;
    const uint64_t g1 = (uint64_t)(blockIdx.x + 1) * p.groups / gridDim.x;
    run_groups<kLife, kTW, kT>(p, lay, in, out, g0, g1, 1, smem, keep, rot, it, p.rec[0], p.rec[1],
                               p.mode == 1u);
  }
  bulk_wait_all();
  settle_abort();
}

// kT steps (1, 2, 4 or 8) of many instances (each with its own fractal, level
// and buffers) that share one tile-row instantiation, in a single persistent
// launch.  parity selects the launch's input: buffer 0 or buffer 1 (and the
// border records of that buffer); mode 1 writes only the input's records
// (before the first step of a run), mode 2 (one step per launch) gathers the
// halo from the state instead of the records and writes the output's.  CTA c
// walks its schedule entries, each a run of groups of one instance (g_first,
// g_first + g_stride, ... below g_end); the instance's description is copied
// to shared memory for the run (its fields are read throughout the group
// loop).
template <bool kLife, int kTW, int kT>
__global__ void __launch_bounds__(kTiledMaxThreads, 3) step_batch_kernel(
    const TiledDev *__restrict__ devs, uint8_t *const *__restrict__ buf0,
    uint8_t *const *__restrict__ buf1, const BatchWork *__restrict__ work,
    const uint32_t *__restrict__ sched_start, TileLayout lay, uint32_t parity, uint32_t mode) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(16) TiledDev s_dev;
  static_assert(sizeof(TiledDev) % 4 == 0, "TiledDev is copied as words");
  uint32_t keep[5], rot[5];
  make_transpose(threadIdx.x & 31u, keep, rot);
  init_barriers(smem, lay);
  uint32_t it = 0;
  for (uint32_t e = sched_start[blockIdx.x]; e < sched_start[blockIdx.x + 1]; ++e) {
    const BatchWork w = work[e];
    __syncthreads();  // every thread is done with the previous entry's description
    const uint32_t *src = reinterpret_cast<const uint32_t *>(devs + w.instance);
    for (uint32_t i = threadIdx.x; i < sizeof(TiledDev) / 4; i += blockDim.x)
      reinterpret_cast<uint32_t *>(&s_dev)[i] = __ldg(src + i);
    __syncthreads();  // s_dev complete: run_groups reads its sizes before its own first barrier
    const uint8_t *in = parity ? buf1[w.instance] : buf0[w.instance];
    uint8_t *out = parity ? buf0[w.instance] : buf1[w.instance];
    run_groups<kLife, kTW, kT>(s_dev, lay, in, out, w.g_first, w.g_end, w.g_stride, smem, keep, rot,
                               it, mode == 0u ? s_dev.rec[parity] : nullptr,
                               s_dev.rec[mode == 1u ? parity : parity ^ 1u], mode == 1u);
  }
  bulk_wait_all();
  settle_abort();
}

// One thread per (direction, tile): the adjacent tile of every tile, computed
// once per fractal and tile level by the carry walk and kept in HBM.
__global__ void build_adjacency_kernel(FracDev f, TiledDev p, uint32_t *__restrict__ adj) {
  __shared__ uint8_t tab[768];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) {
    tab[i] = f.taux[i];
    tab[256 + i] = f.tauy[i];
    tab[512 + i] = f.hnu[i];
  }
  __syncthreads();
  const uint64_t n = (uint64_t)p.ndirs * p.tiles;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t j = (uint32_t)(i / p.tiles);
    uint64_t t = i - (uint64_t)j * p.tiles;
    uint32_t ty = (uint32_t)(t / p.tiles_x), tx = (uint32_t)(t - (uint64_t)ty * p.tiles_x);
    uint32_t d = p.dir_list[j], ntx, nty;
    uint32_t r = ~0u;
    if (adjacent_tile(f, p.L, tab, tab + 256, tab + 512, tx, ty, (int)(d % 3) - 1,
                      (int)(d / 3) - 1, ntx, nty))
      r = nty * p.tiles_x + ntx;
    adj[i] = r;
  }
}

}  // namespace
}  // namespace sq
