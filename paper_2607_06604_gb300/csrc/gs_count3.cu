// Binned triangle counts (Sec. 2.2), GB300 layout. Two kernels give the same
// counts and exact weighted sums:
//
// k_count3p (the default): every triangle i < j < k is found at its smallest
// vertex i from the pair (j, k) of N+(i). The CTA stages the hub-relative
// displacement of every neighbour and tests each pair of N+(i) directly: it
// is an edge exactly when its lattice distance lies in [E_0, E_nb), and the
// bin comes from the same squared distance. No spoke row is read; the work
// is C(|N+(i)|, 2) integer distance tests per hub on shared-memory operands.
//
// k_count3 (the merge-walk of Sec. 3.1): for each hub i and spoke j in N+(i),
// the triangles (i, j, k) with k > j are k in N+(i) intersected with N+(j).
// The paper walks both sorted lists with two pointers; here one persistent
// 1024-thread CTA per SM takes one hub at a time and stages N+(i) in shared
// memory with a bulk (TMA) copy. Because ids are cell ordered, N+(i) lies in
// a short id span above i, so the CTA writes every neighbour's bin into a
// shared byte table indexed by id - (i + 1) (0xFF = not a neighbour). Each
// warp then streams the row N+(j) of one spoke at a time with 128-bit loads
// (four edge words per lane) and probes the table with one subtraction and
// one byte load; a spoke row is abandoned as soon as its ids pass the
// largest id of N+(i) (the merge-walk's exhaustion rule). Only the entries
// written are reset afterwards. Hubs whose span exceeds the table
// (wrap-around neighbours of a periodic box, very sparse catalogues) use a
// shared hash of N+(i) in the same memory, staged in segments.
//
// Both: the configuration index comes from a shared table over (b_ij, b_ik,
// b_jk); counts go to per-CTA shared-memory histograms flushed with one
// 64-bit atomic per bin. Weighted sums use exact fixed point: per hub, 96-bit
// sums of W_j W_k kept in 32-bit limbs, multiplied by W_i into the CTA's
// 128-bit sums, flushed into 192-bit global accumulators.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kThreads = 1024;
constexpr int kWarps = kThreads / 32;
constexpr int kStageCap = 4096;   // hub-row words staged in shared memory
constexpr int kSegCap = 2048;     // hash path: hub-row words per segment
constexpr int kHashMax = 8192;    // hash path: slots, >= 4 x segment words
constexpr int kLutMax = 16384;    // nb^3 entries of the configuration table
constexpr int kRing = 4;          // prefetch ring: 128-word slots per warp
constexpr uint8_t kAbsent = 0xFF;

// One catalogue's arrays. A batched launch carries one per catalogue.
struct Cat {
  const int64_t* __restrict__ ptr;
  const int32_t* __restrict__ deg;
  const uint32_t* __restrict__ adj;  // row j at row_at(adj, ptr, j, adj_off, split, adj_off2)
  int64_t adj_off, split, adj_off2;
  const int64_t* __restrict__ W;   // fixed-point weights (weighted launches)
  unsigned long long* counts;  // [nconf]
  unsigned long long* wacc;    // [nconf][3] 192-bit weighted sums
  int64_t hub_begin, hub_end;
  const int4* __restrict__ xyzp;  // (x, y, z, caller index) in internal order
  int64_t box;                    // periodic side in lattice units, 0 = open box
};

struct Args {
  Cat one;                // single-catalogue launches
  const Cat* cats;        // batched launches: ncats catalogues whose hubs
  const int64_t* base;    // form one queue; base[k] = first queue index of k
  int ncats;
  int nb, nconf;
  int span_cap;           // bytes of the direct-address table (multiple of 16)
  int seg_cap;            // hash path segment (<= kSegCap, multiple of 4)
  int force_hash;         // 1: every hub takes the hash path
  int stage_cap;          // hub rows up to this many words are staged
  int stage_alloc;        // words of the staging buffer
  int use_lut;            // 1: configuration index from the shared table
  int compact;            // 1: weighted hits compacted per warp before recording
  int ring;               // 1: spoke rows prefetched through a per-warp cp.async ring
  uint32_t first_wait_limit;  // polls allowed for a block's first staging wait
  unsigned long long* hub_counter;
  int* err;
};

struct Smem {
  uint8_t* table;      // span_cap bytes; the hash path reuses it as words
  uint32_t* stage;     // stage_alloc words
  int64_t* wst;        // weighted: stage_alloc (W_k, bin(i, k)) pairs of N+(i), 8 bytes each
  uint32_t* queue;     // weighted, compacting launches: 128 hits per warp (or nullptr)
  uint32_t* ring;      // prefetching launches: kRing 128-word slots per warp (or nullptr)
  int* ring_sp;        // the spoke of each slot
  uint16_t* lut;       // nb^3 configuration indices (or nullptr)
  unsigned* hist;      // nconf
  unsigned long long* whist;  // 2 nconf (lo, hi) words: the CTA's 128-bit sums
  unsigned* hacc;      // 3 nconf: the current hub's 96-bit sums of W_j W_k (lo, mid, hi)
};

// LUT: the configuration table is staged (a launch-time choice, compiled in
// so that the arithmetic rank is not carried along on the table path).
template <bool LUT>
__device__ inline int conf_index(const Smem& sm, int bij, int bik, int bjk, int nb) {
  if constexpr (LUT) return (int)sm.lut[(bij * nb + bik) * nb + bjk];
  else return conf3_rank(bij, bik, bjk, nb);
}

// The same with the table row of b_ij precomputed (lbase = b_ij nb^2).
template <bool LUT>
__device__ inline int conf_at(const Smem& sm, int lbase, int bij, int bik, int bjk, int nb) {
  if constexpr (LUT) return (int)sm.lut[lbase + bik * nb + bjk];
  else return conf3_rank(bij, bik, bjk, nb);
}

// Weight modes: kNone and kExact (fixed-point integers: exact 128-bit
// products in shared 128-bit accumulators, 192-bit global sums; shared FP64
// reductions measured slower than this on GB300).
// kExactPos is kExact for weights known to be nonnegative (a cheaper carry
// chain in the per-hub limbs).
enum : int { kNone = 0, kExact = 2, kExactPos = 3 };
template <int WM>
using WType = int64_t;

// One triangle. With shared histograms the weight argument is W_j (the
// spoke's own weight): W_j W_k (|.| < 2^60) is added to the hub's 96-bit
// accumulator with 32-bit shared atomics only (64-bit shared atomics cost
// about 3.5 times as much on GB300), and fold_hub multiplies the hub's sums
// by W_i once per hub. With global histograms it is W_i W_j and the
// 128-bit product goes straight to the 192-bit global sums.
template <int WM, bool SMEM_HIST>
__device__ inline void record(const Smem& sm, const Cat& c, int cf, WType<WM> Wsp, WType<WM> Wk) {
  if (SMEM_HIST) atomicAdd(sm.hist + cf, 1u);
  else atomicAdd(c.counts + cf, 1ull);
  if constexpr (WM >= kExact) {
    if (SMEM_HIST) {
      // |W| < 2^30, so the product is one 32 x 32 -> 64-bit multiply
      const long long x = (long long)(int32_t)Wsp * (int32_t)Wk;
      const uint32_t x0 = (uint32_t)x;
      const uint32_t x1 = (uint32_t)((unsigned long long)x >> 32);
      const uint32_t o0 = atomicAdd(sm.hacc + 3 * cf, x0);
      const uint32_t c0 = (o0 + x0 < o0) ? 1u : 0u;
      const uint32_t a1 = x1 + c0;
      if constexpr (WM == kExactPos) {
        // 0 <= x < 2^60: x1 + c0 cannot wrap and the top limb only takes
        // the mid limb's carries
        const uint32_t o1 = atomicAdd(sm.hacc + 3 * cf + 1, a1);
        if (o1 + a1 < o1) atomicAdd(sm.hacc + 3 * cf + 2, 1u);
      } else {
        uint32_t a2 = (x < 0 ? 0xFFFFFFFFu : 0u) + ((a1 < x1) ? 1u : 0u);
        if (a1) {
          const uint32_t o1 = atomicAdd(sm.hacc + 3 * cf + 1, a1);
          a2 += (o1 + a1 < o1) ? 1u : 0u;
        }
        if (a2) atomicAdd(sm.hacc + 3 * cf + 2, a2);
      }
    } else {
      long long lo, hi;
      mul_i128(Wsp, Wk, &lo, &hi);
      atomic_add_i192(c.wacc + 3 * cf, (unsigned long long)lo, (unsigned long long)hi);
    }
  }
}

template <int WM>
__device__ inline WType<WM> wget(const Cat& c, int64_t k) {
  if constexpr (WM >= kExact) return c.W[k];
  else return 0;
}

// EQUI: equilateral configurations only (all three sides in one bin, the
// configurations (b, b, b)): words of N+(j) in another bin than b_ij are not
// probed, hits need b_ik = b_ij, and the histograms have nb entries.
template <int WM, bool SMEM_HIST, bool BATCH, bool LUT, bool EQUI = false>
__global__ void __launch_bounds__(kThreads, 1) k_count3(Args a) {
  constexpr bool WEIGHTED = WM != kNone;
  using WT = WType<WM>;
  extern __shared__ __align__(16) unsigned char smem[];
  Smem sm;
  {
    unsigned char* p = smem;
    sm.table = p;
    p += a.span_cap;
    sm.stage = reinterpret_cast<uint32_t*>(p);
    p += (size_t)a.stage_alloc * 4;
    sm.wst = reinterpret_cast<int64_t*>(p);
    if (WEIGHTED) p += (size_t)a.stage_alloc * 8;
    sm.queue = (WEIGHTED && a.compact) ? reinterpret_cast<uint32_t*>(p) : nullptr;
    if (WEIGHTED && a.compact) p += (size_t)kWarps * 128 * 4;
    sm.ring = a.ring ? reinterpret_cast<uint32_t*>(p) : nullptr;
    if (a.ring) p += (size_t)kWarps * kRing * 128 * 4;
    sm.ring_sp = a.ring ? reinterpret_cast<int*>(p) : nullptr;
    if (a.ring) p += (size_t)kWarps * kRing * 4;
    const int nb3 = a.nb * a.nb * a.nb;
    sm.lut = (a.use_lut && nb3 <= kLutMax) ? reinterpret_cast<uint16_t*>(p) : nullptr;
    if (a.use_lut && nb3 <= kLutMax) p += ((nb3 * 2 + 15) / 16) * 16;
    sm.hist = reinterpret_cast<unsigned*>(p);
    p += ((a.nconf * 4 + 15) / 16) * 16;
    sm.whist = reinterpret_cast<unsigned long long*>(p);
    sm.hacc = reinterpret_cast<unsigned*>(sm.whist + 2 * a.nconf);
  }
  __shared__ uint64_t bar;
  __shared__ int64_t s_hub;
  __shared__ unsigned long long s_pending;
  __shared__ int s_flush, s_cat, s_cur, s_next;
  __shared__ int s_warp_sum[kWarps];
  __shared__ unsigned long long s_red[kWarps];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nb = a.nb;
  // idle table: all bytes 0xFF (byte table) or all bits clear (weighted bitmap)
  const uint32_t idle = WEIGHTED ? 0u : kSentinel;
  for (int k = tid; k < a.span_cap / 4; k += kThreads) reinterpret_cast<uint32_t*>(sm.table)[k] = idle;
  if (sm.lut)
    for (int k = tid; k < nb * nb * nb; k += kThreads)
      sm.lut[k] = (uint16_t)conf3_rank(k / (nb * nb), (k / nb) % nb, k % nb, nb);
  if (SMEM_HIST) {
    for (int k = tid; k < a.nconf; k += kThreads) sm.hist[k] = 0;
    if (WEIGHTED)
      for (int k = tid; k < (WM >= kExact ? 2 : 1) * a.nconf; k += kThreads) sm.whist[k] = 0;
    if (WM >= kExact)
      for (int k = tid; k < 3 * a.nconf; k += kThreads) sm.hacc[k] = 0;
  }
  if (tid == 0) {
    mbar_init(&bar, 1);
    s_pending = 0;
    s_cur = BATCH ? -1 : 0;
  }
  __syncthreads();
  uint32_t phase = 0;
  Cat c = a.one;
  int cur = BATCH ? -1 : 0;

  // shared histograms -> the current catalogue's global ones
  auto flush = [&]() {
    if (!SMEM_HIST || cur < 0) return;
    for (int k = tid; k < a.nconf; k += kThreads) {
      const unsigned v = sm.hist[k];
      if (v) {
        atomicAdd(c.counts + k, (unsigned long long)v);
        sm.hist[k] = 0;
      }
      if (WM >= kExact) {
        const unsigned long long lo = sm.whist[2 * k], hi = sm.whist[2 * k + 1];
        if (lo | hi) {
          atomic_add_i192(c.wacc + 3 * k, lo, hi);
          sm.whist[2 * k] = sm.whist[2 * k + 1] = 0;
        }
      }
    }
  };
  // the hub's 96-bit sums S[k] of W_j W_k, times W_i, into the CTA's
  // 128-bit sums (each thread owns its configurations; no atomics)
  auto fold_hub = [&](int64_t Wi) {
    if constexpr (SMEM_HIST && WM >= kExact) {
      for (int k = tid; k < a.nconf; k += kThreads) {
        const uint32_t l = sm.hacc[3 * k], m = sm.hacc[3 * k + 1], h = sm.hacc[3 * k + 2];
        if (!(l | m | h)) continue;
        sm.hacc[3 * k] = sm.hacc[3 * k + 1] = sm.hacc[3 * k + 2] = 0u;
        // S = (int32)h 2^64 + ml; S W_i as a 128-bit two's-complement value
        const unsigned long long ml = ((unsigned long long)m << 32) | l;
        const unsigned long long uw = (unsigned long long)Wi;
        const unsigned long long plo = ml * uw;
        unsigned long long phi = __umul64hi(ml, uw) - (Wi < 0 ? ml : 0ull);
        phi += (unsigned long long)((long long)(int32_t)h * Wi);
        const unsigned long long olo = sm.whist[2 * k];
        const unsigned long long nlo = olo + plo;
        sm.whist[2 * k] = nlo;
        sm.whist[2 * k + 1] += phi + ((nlo < olo) ? 1ull : 0ull);
      }
    }
  };

  // bounded wait on the bulk copy; false when it timed out (block-uniform)
  // On an expired wait the block reports it, then waits (bounded again) for
  // its own copy to land before giving up, so no copy outlives the block.
  // a.first_wait_limit replaces the first wait's budget (tests use 0).
  uint32_t wait_budget = a.first_wait_limit;
  auto wait_stage = [&]() -> bool {
    const bool ok = mbar_wait(&bar, phase, wait_budget);
    wait_budget = kWaitLimit;
    if (__syncthreads_or(!ok)) {
      if (tid == 0) atomicOr(a.err, kErrTimeout);
      if (!ok) mbar_wait(&bar, phase, kWaitLimit);
      __syncthreads();
      return false;
    }
    phase ^= 1u;
    return true;
  };

  for (;;) {
    if (tid == 0) {
      const int64_t q = (int64_t)atomicAdd(a.hub_counter, 1ull);
      int k = 0;
      int64_t hub;
      bool valid;
      if (BATCH) {
        valid = q < a.base[a.ncats];
        if (valid) {
          int lo = 0, hi = a.ncats;  // largest k with base[k] <= q
          while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (a.base[mid] <= q) lo = mid;
            else hi = mid;
          }
          k = lo;
        }
        hub = valid ? q - a.base[k] : 0;
      } else {
        hub = a.one.hub_begin + q;
        valid = hub < a.one.hub_end;
      }
      s_hub = valid ? hub : -1;
      s_cat = k;
      s_flush = 0;
      s_next = 0;
      if (valid) {
        const int32_t* dg = BATCH ? a.cats[k].deg : a.one.deg;
        const unsigned long long d = (unsigned long long)dg[hub];
        const unsigned long long need = d * (d - (d > 0)) / 2;  // triangles at i <= C(d,2)
        if (k != s_cur || s_pending + need > 0xFFFFFFFFull) {
          s_flush = 1;
          s_pending = need;
          s_cur = k;
        } else {
          s_pending += need;
        }
      }
    }
    __syncthreads();
    const int64_t i = s_hub;
    if (i < 0) break;
    if (s_flush) {
      flush();
      __syncthreads();
    }
    if (BATCH && s_cat != cur) {
      cur = s_cat;
      c = a.cats[cur];
    }
    const int d = c.deg[i];
    if (d < 2) {
      __syncthreads();
      continue;
    }
    const uint32_t* row = row_at(c.adj, c.ptr, i, c.adj_off, c.split, c.adj_off2);
    const WT Wi = wget<WM>(c, i);
    // staged (W_k, bin(i, k)) pairs: one 64-bit load per hit, |W_k| < 2^30
    int2* wst2 = reinterpret_cast<int2*>(sm.wst);
    const uint32_t hub_hi = edge_id(row[d - 1]);
    const int64_t span = (int64_t)hub_hi - i;  // ids i+1 .. hub_hi
    const bool staged = d <= a.stage_cap;
    // weighted hubs need their row and weights staged (positions come from
    // the bitmap rank); each 32 ids take one 64-bit entry: the bitmap word
    // and the rank of its first bit, read together by one shared load
    const int64_t table_span = WEIGHTED ? (int64_t)(a.span_cap / 8) * 32 : (int64_t)a.span_cap;
    bool use_table = !a.force_hash && (!WEIGHTED || staged);
    // The table covers ids [i+1, near_hi] at offsets 0 .. len1-1 and, for
    // rows split at their largest id gap (wrap-around neighbours of a
    // periodic box), [far_lo, hub_hi] after them.
    uint32_t near_hi = hub_hi, far_lo = hub_hi + 1u;
    int64_t len1 = span, tspan = span;
    const uint32_t* hr = row;
    if (use_table) {
      if (staged) {
        if (tid == 0) bulk_load(sm.stage, row, (uint32_t)pad_row(d) * 4u, &bar);
        // weighted: staged word = 256 W_k + bin(i, k), one load per hit
        if (WEIGHTED)
          for (int k = tid; k < d; k += kThreads) {
            const uint32_t w = row[k];
            wst2[k] = make_int2((int)wget<WM>(c, edge_id(w)), (int)edge_bin(w));
          }
        if (!wait_stage()) return;
        hr = sm.stage;
      }
      if (span > table_span) {
        // largest gap between consecutive neighbour ids (first one on ties)
        unsigned long long best = 0ull;
        for (int k = tid; k < d - 1; k += kThreads) {
          const unsigned long long gap = edge_id(hr[k + 1]) - edge_id(hr[k]);
          const unsigned long long key = (gap << 32) | (0xFFFFFFFFull - (unsigned long long)k);
          best = best > key ? best : key;
        }
        for (int o = 16; o; o >>= 1) {
          const unsigned long long y = __shfl_xor_sync(0xffffffffu, best, o);
          best = best > y ? best : y;
        }
        if (lane == 0) s_red[warp] = best;
        __syncthreads();
        if (warp == 0) {
          best = s_red[lane];
          for (int o = 16; o; o >>= 1) {
            const unsigned long long y = __shfl_xor_sync(0xffffffffu, best, o);
            best = best > y ? best : y;
          }
          if (lane == 0) s_red[0] = best;
        }
        __syncthreads();
        const int ks = (int)(0xFFFFFFFFull - (s_red[0] & 0xFFFFFFFFull));
        __syncthreads();
        near_hi = edge_id(hr[ks]);
        far_lo = edge_id(hr[ks + 1]);
        len1 = (int64_t)near_hi - i;
        tspan = len1 + ((int64_t)hub_hi - far_lo + 1);
        use_table = tspan <= table_span;
      }
    }
    if (use_table) {
      // ---------------- direct-address table path
      const uint32_t base = (uint32_t)(i + 1);
      const uint32_t far_off = (uint32_t)len1;
      auto slot = [&](uint32_t key) -> uint32_t {
        return key <= near_hi ? key - base : key - far_lo + far_off;
      };
      uint2* bm = reinterpret_cast<uint2*>(sm.table);  // (bits, rank of bit 0)
      const int nw = (int)((tspan + 31) >> 5);
      if (WEIGHTED) {
        for (int k = tid; k < d; k += kThreads) {
          const uint32_t off = slot(edge_id(hr[k]));
          atomicOr(&bm[off >> 5].x, 1u << (off & 31));
        }
        __syncthreads();
        // exclusive prefix of the words' popcounts: the rank of every bit
        const int per = (nw + kThreads - 1) / kThreads;
        const int w0 = min(nw, tid * per), w1 = min(nw, w0 + per);
        int sum = 0;
        for (int q = w0; q < w1; ++q) sum += __popc(bm[q].x);
        int x = sum;
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, x, o);
          if (lane >= o) x += y;
        }
        if (lane == 31) s_warp_sum[warp] = x;
        __syncthreads();
        if (warp == 0) {
          int t = s_warp_sum[lane];
          for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
          }
          s_warp_sum[lane] = t;
        }
        __syncthreads();
        int run = x - sum + (warp ? s_warp_sum[warp - 1] : 0);
        for (int q = w0; q < w1; ++q) {
          bm[q].y = (uint32_t)run;
          run += __popc(bm[q].x);
        }
      } else {
        for (int k = tid; k < d; k += kThreads) {
          const uint32_t w = hr[k];
          sm.table[slot(edge_id(w))] = (uint8_t)edge_bin(w);
        }
      }
      __syncthreads();
      // Each warp walks spoke rows in 128-word chunks. By default the next
      // chunk, or the first chunk of the warp's next spoke, is loaded into
      // registers before the current one is probed.
      const uint4 none = make_uint4(kSentinel, kSentinel, kSentinel, kSentinel);
      const bool split = far_lo <= hub_hi;  // two table ranges (block-uniform)
      uint32_t* wq = sm.queue ? sm.queue + warp * 128 : nullptr;
      // probes and hits of one 128-word chunk (four edge words per lane) of
      // a spoke row whose hub edge has bin bij
      auto process = [&](const uint4 v, const int bij, const int lbase, const WT Wsp) {
        const uint32_t vv[4] = {v.x, v.y, v.z, v.w};
        // all four probes are issued before any hit is handled, so their
        // shared-memory latencies overlap; keys past the hub row probe
        // slot 0 and are discarded
        bool ok[4];
        uint32_t off[4];
        if (split) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const uint32_t key = edge_id(vv[q]);
            ok[q] = key <= hub_hi && (key <= near_hi || key >= far_lo) &&
                    (!EQUI || edge_bin(vv[q]) == (uint32_t)bij);
            off[q] = ok[q] ? slot(key) : 0u;
          }
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const uint32_t key = edge_id(vv[q]);
            ok[q] = key <= hub_hi && (!EQUI || edge_bin(vv[q]) == (uint32_t)bij);
            off[q] = ok[q] ? key - base : 0u;
          }
        }
        if (WEIGHTED) {
          uint2 bw[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) bw[q] = bm[off[q] >> 5];
          if (wq) {
            // compact the chunk's hits into the warp's queue, then record
            // them one per lane (full lanes instead of four divergent passes)
            int n = 0;
            const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const uint32_t bit = 1u << (off[q] & 31);
              const bool hit = ok[q] && (bw[q].x & bit);
              const uint32_t m = __ballot_sync(0xffffffffu, hit);
              if (hit)
                wq[n + __popc(m & lt)] =
                    (bw[q].y + (uint32_t)__popc(bw[q].x & (bit - 1u))) | (edge_bin(vv[q]) << 16);
              n += __popc(m);
            }
            __syncwarp();
            for (int r = lane; r < n; r += 32) {
              const uint32_t e = wq[r];
              const int2 pk = wst2[e & 0xFFFFu];
              if (!EQUI || pk.y == bij)
                record<WM, SMEM_HIST>(
                    sm, c, EQUI ? bij : conf_at<LUT>(sm, lbase, bij, pk.y, (int)(e >> 16), nb), Wsp,
                    (WT)pk.x);
            }
            __syncwarp();
          } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const uint32_t bit = 1u << (off[q] & 31);
              if (ok[q] && (bw[q].x & bit)) {
                const int pos = (int)bw[q].y + __popc(bw[q].x & (bit - 1u));
                const int2 pk = wst2[pos];
                if (!EQUI || pk.y == bij)
                  record<WM, SMEM_HIST>(
                      sm, c,
                      EQUI ? bij : conf_at<LUT>(sm, lbase, bij, pk.y, (int)edge_bin(vv[q]), nb),
                      Wsp, (WT)pk.x);
              }
            }
          }
        } else {
          uint8_t bik[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) bik[q] = sm.table[off[q]];
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (ok[q] && bik[q] != kAbsent && (!EQUI || bik[q] == bij))
              record<WM, SMEM_HIST>(
                  sm, c, EQUI ? bij : conf_at<LUT>(sm, lbase, bij, bik[q], (int)edge_bin(vv[q]), nb),
                  WT(0), WT(0));
        }
      };
      if (sm.ring) {
        // Spoke rows through a per-warp ring of kRing 128-word slots filled by
        // asynchronous copies (cp.async, 16 bytes per lane), so kRing - 1
        // chunks are in flight while one is processed. The chunk stream runs
        // through the warp's spokes in order; chunks already issued for a
        // spoke that the walk has abandoned (its ids passed hub_hi) are
        // skipped. Each lane copies and later reads its own 16 bytes of a
        // slot; the slot's spoke index is written by lane 0.
        uint32_t* ring = sm.ring + (size_t)warp * kRing * 128;
        int* rsp = sm.ring_sp + warp * kRing;
        int psp = d, pdj4 = 0, pt0 = 0, dead = -1;
        const uint32_t* prj = nullptr;
        auto next_spoke = [&]() {
          int q = 0;
          if (lane == 0) q = atomicAdd(&s_next, 1);
          q = __shfl_sync(0xffffffffu, q, 0);
          psp = q;
          pt0 = 0;
          if (q < d - 1) {
            const uint32_t w = hr[q];
            prj = row_at(c.adj, c.ptr, edge_id(w), c.adj_off, c.split, c.adj_off2);
            pdj4 = (int)pad_row(c.deg[edge_id(w)]);
          }
        };
        auto produce = [&](int st) {
          while (psp < d - 1 && (pt0 >= pdj4 || psp == dead)) next_spoke();
          uint32_t* dst = ring + st * 128 + lane * 4;
          if (psp < d - 1) {
            const int t = pt0 + lane * 4;
            if (t < pdj4) cp_async16(dst, prj + t);
            else *reinterpret_cast<uint4*>(dst) = none;
            pt0 += 128;
          }
          if (lane == 0) rsp[st] = psp < d - 1 ? psp : -1;
          cp_async_commit();
        };
        next_spoke();
        for (int st = 0; st < kRing - 1; ++st) produce(st);
        int csp = -1, bij = 0, lbase = 0;
        WT Wsp = 0;
        for (int it = 0;; ++it) {
          produce((it + kRing - 1) % kRing);
          cp_async_wait<kRing - 1>();
          __syncwarp();
          const int st = it % kRing;
          const int sp = rsp[st];
          if (sp < 0) break;
          const uint4 v = *reinterpret_cast<const uint4*>(ring + st * 128 + lane * 4);
          if (sp != dead) {
            if (sp != csp) {
              csp = sp;
              const uint32_t wij = hr[sp];
              bij = (int)edge_bin(wij);
              lbase = bij * nb * nb;
              if (WEIGHTED) {
                const WT Wj = staged ? (WT)wst2[sp].x : wget<WM>(c, edge_id(wij));
                Wsp = SMEM_HIST ? Wj : Wi * Wj;
              }
            }
            process(v, bij, lbase, Wsp);
            const uint32_t last = __shfl_sync(0xffffffffu, v.w, 31);
            if (edge_id(last) > hub_hi) dead = sp;
          }
          __syncwarp();
        }
        cp_async_wait_all();
        __syncwarp();
      } else {
        int sp = 0;
        if (lane == 0) sp = atomicAdd(&s_next, 1);
        sp = __shfl_sync(0xffffffffu, sp, 0);
        if (sp < d - 1) {  // the last neighbour has no k above it
          uint32_t wij = hr[sp];
          const uint32_t* rj = row_at(c.adj, c.ptr, edge_id(wij), c.adj_off, c.split, c.adj_off2);
          int dj4 = (int)pad_row(c.deg[edge_id(wij)]);
          int t0 = 0;
          uint4 v = (lane * 4 < dj4) ? ldg_nc_v4(rj + lane * 4) : none;
          // per-spoke constants: b_ij, the spoke's weight factor, and the row of
          // the configuration table that b_ij selects
          int bij = (int)edge_bin(wij);
          int lbase = bij * nb * nb;
          WT Wsp = 0;
          if (WEIGHTED) {
            const WT Wj = staged ? (WT)wst2[sp].x : wget<WM>(c, edge_id(wij));
            Wsp = SMEM_HIST ? Wj : Wi * Wj;
          }
          for (;;) {
            const uint32_t last = __shfl_sync(0xffffffffu, v.w, 31);
            const bool more = edge_id(last) <= hub_hi && t0 + 128 < dj4;
            uint4 vn = none;
            int nsp = sp;
            uint32_t nwij = wij;
            const uint32_t* nrj = rj;
            int ndj4 = dj4;
            if (more) {
              const int t = t0 + 128 + lane * 4;
              vn = (t < dj4) ? ldg_nc_v4(rj + t) : none;
            } else {
              if (lane == 0) nsp = atomicAdd(&s_next, 1);
              nsp = __shfl_sync(0xffffffffu, nsp, 0);
              if (nsp < d - 1) {
                nwij = hr[nsp];
                nrj = row_at(c.adj, c.ptr, edge_id(nwij), c.adj_off, c.split, c.adj_off2);
                ndj4 = (int)pad_row(c.deg[edge_id(nwij)]);
                vn = (lane * 4 < ndj4) ? ldg_nc_v4(nrj + lane * 4) : none;
              }
            }
            process(v, bij, lbase, Wsp);
            if (more) {
              t0 += 128;
            } else {
              if (nsp >= d - 1) break;
              sp = nsp;
              wij = nwij;
              rj = nrj;
              dj4 = ndj4;
              t0 = 0;
              bij = (int)edge_bin(wij);
              lbase = bij * nb * nb;
              if (WEIGHTED) {
                const WT Wj = staged ? (WT)wst2[sp].x : wget<WM>(c, edge_id(wij));
                Wsp = SMEM_HIST ? Wj : Wi * Wj;
              }
            }
            v = vn;
          }
        }
      }
      __syncthreads();
      fold_hub(Wi);
      if (WEIGHTED) {
        // ranks are rewritten for every word a hub uses; only bits need clearing
        for (int k = tid; k < d; k += kThreads) bm[slot(edge_id(hr[k])) >> 5].x = 0u;
      } else {
        for (int k = tid; k < d; k += kThreads) sm.table[slot(edge_id(hr[k]))] = kAbsent;
      }
      __syncthreads();
      continue;
    }
    // ---------------- hash path (span wider than the table)
    uint32_t* table = reinterpret_cast<uint32_t*>(sm.table);
    const int tcap_bits = [&] {
      int b = 7;
      while ((2 << b) * 4 <= a.span_cap && b < 13) ++b;
      return b;
    }();
    const int seg_cap = min(a.seg_cap, (1 << tcap_bits) / 4);
    for (int s0 = 0; s0 < d; s0 += seg_cap) {
      const int sn = min(seg_cap, d - s0);
      const int sn4 = (int)pad_row(sn);
      if (tid == 0) bulk_load(sm.stage, row + s0, (uint32_t)sn4 * 4u, &bar);
      int tbits = 7;
      while ((1 << tbits) < 4 * sn && tbits < tcap_bits) ++tbits;
      const int T = 1 << tbits;
      const int shift = 32 - tbits;
      if (WEIGHTED)
        for (int k = tid; k < T; k += kThreads) table[k] = kSentinel;
      if (!wait_stage()) return;
      for (int k = tid; k < sn; k += kThreads) {
        const uint32_t w = sm.stage[k];
        uint32_t h = (edge_id(w) * kHashMul) >> shift;
        while (atomicCAS(table + h, kSentinel, w) != kSentinel) h = (h + 1) & (T - 1);
      }
      __syncthreads();
      const uint32_t seg_lo = edge_id(sm.stage[0]);
      const uint32_t seg_hi = edge_id(sm.stage[sn - 1]);
      for (int sp = warp; sp < d; sp += kWarps) {
        const uint32_t wij = (d <= seg_cap) ? sm.stage[sp] : row[sp];
        const uint32_t j = edge_id(wij);
        if (j >= seg_hi) break;  // every k > j; none left in this segment
        const int bij = (int)edge_bin(wij);
        const WT Wj = wget<WM>(c, j);
        const WT Wsp = SMEM_HIST ? Wj : Wi * Wj;
        const uint32_t* rj = row_at(c.adj, c.ptr, j, c.adj_off, c.split, c.adj_off2);
        const int dj4 = (int)pad_row(c.deg[j]);
        int start = 0;
        if (s0 > 0) {  // skip to the first id >= seg_lo (rows are sorted)
          int lo = 0, hi = c.deg[j];
          const uint32_t key = seg_lo << 8;
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (rj[mid] < key) lo = mid + 1;
            else hi = mid;
          }
          start = lo & ~3;
        }
        for (int t0 = start; t0 < dj4; t0 += 128) {
          const int t = t0 + lane * 4;
          const uint4 v = (t < dj4) ? ldg_nc_v4(rj + t)
                                    : make_uint4(kSentinel, kSentinel, kSentinel, kSentinel);
          const uint32_t vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const uint32_t key = edge_id(vv[q]);
            if (key > seg_hi || (EQUI && edge_bin(vv[q]) != (uint32_t)bij)) continue;
            uint32_t h = (key * kHashMul) >> shift;
            for (;;) {
              const uint32_t e = table[h];
              if (e == kSentinel) break;
              if (edge_id(e) == key) {
                if (!EQUI || (int)edge_bin(e) == bij)
                  record<WM, SMEM_HIST>(
                      sm, c,
                      EQUI ? bij
                           : conf_index<LUT>(sm, bij, (int)edge_bin(e), (int)edge_bin(vv[q]), nb),
                      Wsp, wget<WM>(c, key));
                break;
              }
              h = (h + 1) & (T - 1);
            }
          }
          const uint32_t last = __shfl_sync(0xffffffffu, v.w, 31);
          if (edge_id(last) > seg_hi) break;
        }
      }
      __syncthreads();
      // restore the idle table for the next hub
      for (int k = tid; k < T; k += kThreads) table[k] = idle;
      __syncthreads();
    }
    fold_hub(Wi);
  }
  __syncthreads();
  flush();
}


// The instantiation of k_count3 for a launch: weight mode (nonnegative
// weights take the cheaper carry chain), shared or global histograms,
// single or batched, staged configuration table or arithmetic ranks.
template <bool BATCH>
void (*pick_count3(int wm, bool nonneg, bool smem_hist, bool lut))(Args) {
#define GS_K(W, S) (lut ? k_count3<W, S, BATCH, true> : k_count3<W, S, BATCH, false>)
  if (wm == kNone) return smem_hist ? GS_K(kNone, true) : GS_K(kNone, false);
  if (!smem_hist) return GS_K(kExact, false);
  return nonneg ? GS_K(kExactPos, true) : GS_K(kExact, true);
#undef GS_K
}

void (*pick_equi3(int wm, bool nonneg, bool smem_hist))(Args) {
  if (wm == kNone)
    return smem_hist ? k_count3<kNone, true, false, false, true>
                     : k_count3<kNone, false, false, false, true>;
  if (!smem_hist) return k_count3<kExact, false, false, false, true>;
  return nonneg ? k_count3<kExactPos, true, false, false, true>
                : k_count3<kExact, true, false, false, true>;
}

// ----------------------------------------------------------------------------
// Pair-geometry triangle counting (the default launch).
//
// Every triangle i < j < k has j and k in N+(i). The walk above finds the
// pairs (j, k) of N+(i) that are edges by intersecting sorted rows; this
// kernel tests the pairs directly. The CTA stages, for every neighbour of
// the hub, its minimum-image displacement D from the hub (exact lattice
// integers) and the hub edge's bin; then every pair (j, k) of N+(i) with
// j < k is an edge exactly when E_0^2 <= |D_k - D_j|^2 < E_nb^2 (in a
// periodic box 4 E_nb < L makes D_k - D_j the minimum image of k - j), and
// its bin follows from the same squared distance. No spoke row is read:
// the work per hub is C(d, 2) integer distance tests on shared-memory
// operands, and a hit is recorded exactly as in the walk (per-CTA 32-bit
// histograms, per-hub 96-bit sums of W_j W_k folded by W_i).
constexpr int kPThreads = 512;
constexpr int kPBucketMax = 2048;         // buckets no wider than the narrowest bin
constexpr int kPBucketExactMax = 16384;  // buckets that each hold one bin

// Shared-memory updates on 32-bit shared addresses, done only when pred
// holds (no branch): the pair kernel records every examined pair's update
// under its hit predicate, so the warp never diverges on a hit.
__device__ inline void red_add_shared_if(uint32_t a, uint32_t v, bool pred) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %2, 0;\n\t"
      "@p red.shared.add.u32 [%0], %1;\n\t}" ::"r"(a),
      "r"(v), "r"((uint32_t)pred)
      : "memory");
}
__device__ inline uint32_t atom_add_shared_if(uint32_t a, uint32_t v, bool pred) {
  uint32_t old = 0u;  // stays 0 when pred is false
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %3, 0;\n\t"
      "@p atom.shared.add.u32 %0, [%1], %2;\n\t}"
      : "+r"(old)
      : "r"(a), "r"(v), "r"((uint32_t)pred)
      : "memory");
  return old;
}

// One pair's count and, weighted, W_j W_k into the hub's 96-bit limbs
// (hist and hacc as shared addresses), when hit holds.
template <int WM>
__device__ inline void record_if(uint32_t hist, uint32_t hacc, int cf, bool hit, int32_t Wj,
                                 int32_t Wk) {
  red_add_shared_if(hist + 4u * (uint32_t)cf, 1u, hit);
  if constexpr (WM >= kExact) {
    const long long x = (long long)Wj * Wk;
    const uint32_t x0 = (uint32_t)x;
    const uint32_t x1 = (uint32_t)((unsigned long long)x >> 32);
    const uint32_t lo = hacc + 12u * (uint32_t)cf;
    const uint32_t o0 = atom_add_shared_if(lo, x0, hit);
    const uint32_t a1 = x1 + ((o0 + x0 < o0) ? 1u : 0u);
    if constexpr (WM == kExactPos) {
      // 0 <= x < 2^60: x1 + carry cannot wrap; the top limb only takes the
      // mid limb's carries
      const uint32_t o1 = atom_add_shared_if(lo + 4u, a1, hit);
      red_add_shared_if(lo + 8u, 1u, hit && (o1 + a1 < o1));
    } else {
      uint32_t a2 = (x < 0 ? 0xFFFFFFFFu : 0u) + ((a1 < x1) ? 1u : 0u);
      const uint32_t o1 = atom_add_shared_if(lo + 4u, a1, hit && a1 != 0u);
      a2 += (o1 + a1 < o1) ? 1u : 0u;
      red_add_shared_if(lo + 8u, a2, hit && a2 != 0u);
    }
  }
}

struct PArgs {
  Cat one;              // single-catalogue launches
  const Cat* cats;      // batched launches (catalogues with equal bin edges)
  const int64_t* base;
  int ncats;
  int nb, nconf;
  int cap;              // neighbours staged in shared memory
  int use_lut;
  int bk_shift, bk_n;   // squared-distance buckets (bk_n = 0: binary search)
  const int64_t* e2g;   // nb + 1 squared bin edges
  unsigned char* gscratch;  // hubs above cap: per-CTA staging in global memory
  size_t gstride;
  unsigned long long* hub_counter;
  float lin_c;          // linear bins: 1 / m, raised by 2^-20 (see the pair test)
};

__device__ inline int64_t min_image(int64_t d, int64_t box) {
  if (box) {
    if (2 * d >= box) d -= box;
    else if (2 * d < -box) d += box;
  }
  return d;
}

// Binning of a pair's squared distance D2 in the pair kernel.
enum : int {
  kBinSearch = 0,  // range test, then buckets finished by one comparison (or a search)
  kBinTable = 1,   // every squared edge is a multiple of the bucket width: one lookup
  kBinLinear = 2   // E_b = b m 2^t, E_0 = 0: the bin is floor(sqrt(D2 / 2^2t) / m)
};

template <int WM, bool BATCH, bool LUT, int BIN>
__global__ void __launch_bounds__(kPThreads, 2) k_count3p(PArgs a) {
  constexpr bool WEIGHTED = WM != kNone;
  using WT = WType<WM>;
  extern __shared__ __align__(16) unsigned char smem[];
  const int nb = a.nb;
  Smem sm;
  int4* s_stage;
  int64_t* s_e2;
  uint8_t* s_bk;
  {
    unsigned char* p = smem;
    s_stage = reinterpret_cast<int4*>(p);
    p += (size_t)a.cap * 16;
    s_e2 = reinterpret_cast<int64_t*>(p);
    p += (size_t)(nb + 1) * 8;
    p = reinterpret_cast<unsigned char*>(((uintptr_t)p + 15) & ~(uintptr_t)15);
    const int nb3 = nb * nb * nb;
    sm.lut = LUT ? reinterpret_cast<uint16_t*>(p) : nullptr;
    if (LUT) p += ((nb3 * 2 + 15) / 16) * 16;
    sm.hist = reinterpret_cast<unsigned*>(p);
    p += ((a.nconf * 4 + 15) / 16) * 16;
    sm.whist = reinterpret_cast<unsigned long long*>(p);
    sm.hacc = reinterpret_cast<unsigned*>(sm.whist + 2 * a.nconf);
    if (WEIGHTED) p += (size_t)a.nconf * 28;
    s_bk = reinterpret_cast<uint8_t*>(p);
    sm.table = nullptr;
    sm.stage = nullptr;
    sm.wst = nullptr;
    sm.queue = nullptr;
    sm.ring = nullptr;
    sm.ring_sp = nullptr;
  }
  __shared__ int64_t s_hub;
  __shared__ unsigned long long s_pending;
  __shared__ int s_flush, s_cat, s_cur, s_next;

  const int tid = threadIdx.x, lane = tid & 31;
  if (LUT)
    for (int k = tid; k < nb * nb * nb; k += kPThreads)
      sm.lut[k] = (uint16_t)conf3_rank(k / (nb * nb), (k / nb) % nb, k % nb, nb);
  for (int k = tid; k < a.nconf; k += kPThreads) sm.hist[k] = 0;
  if (WEIGHTED) {
    for (int k = tid; k < 2 * a.nconf; k += kPThreads) sm.whist[k] = 0;
    for (int k = tid; k < 3 * a.nconf; k += kPThreads) sm.hacc[k] = 0;
  }
  for (int b = tid; b <= nb; b += kPThreads) s_e2[b] = a.e2g[b];
  for (int k = tid; BIN != kBinLinear && k < a.bk_n; k += kPThreads) {
    const int64_t x = (int64_t)k << a.bk_shift;
    int b = 0;
    while (b + 1 < nb && a.e2g[b + 1] <= x) ++b;
    s_bk[k] = (BIN == kBinTable && x < a.e2g[0]) ? (uint8_t)0xFF : (uint8_t)b;
  }
  if (tid == 0) {
    s_pending = 0;
    s_cur = BATCH ? -1 : 0;
  }
  __syncthreads();
  const int64_t e2lo = s_e2[0], e2hi = s_e2[nb];
  const uint8_t* bk = (BIN != kBinLinear && a.bk_n) ? s_bk : nullptr;
  Cat c = a.one;
  int cur = BATCH ? -1 : 0;

  auto flush = [&]() {
    if (cur < 0) return;
    for (int k = tid; k < a.nconf; k += kPThreads) {
      const unsigned v = sm.hist[k];
      if (v) {
        atomicAdd(c.counts + k, (unsigned long long)v);
        sm.hist[k] = 0;
      }
      if (WEIGHTED) {
        const unsigned long long lo = sm.whist[2 * k], hi = sm.whist[2 * k + 1];
        if (lo | hi) {
          atomic_add_i192(c.wacc + 3 * k, lo, hi);
          sm.whist[2 * k] = sm.whist[2 * k + 1] = 0;
        }
      }
    }
  };
  // the hub's 96-bit sums of W_j W_k, times W_i, into the CTA's 128-bit sums
  auto fold_hub = [&](int64_t Wi) {
    if constexpr (WEIGHTED) {
      for (int k = tid; k < a.nconf; k += kPThreads) {
        const uint32_t l = sm.hacc[3 * k], m = sm.hacc[3 * k + 1], h = sm.hacc[3 * k + 2];
        if (!(l | m | h)) continue;
        sm.hacc[3 * k] = sm.hacc[3 * k + 1] = sm.hacc[3 * k + 2] = 0u;
        const unsigned long long ml = ((unsigned long long)m << 32) | l;
        const unsigned long long uw = (unsigned long long)Wi;
        const unsigned long long plo = ml * uw;
        unsigned long long phi = __umul64hi(ml, uw) - (Wi < 0 ? ml : 0ull);
        phi += (unsigned long long)((long long)(int32_t)h * Wi);
        const unsigned long long olo = sm.whist[2 * k];
        const unsigned long long nlo = olo + plo;
        sm.whist[2 * k] = nlo;
        sm.whist[2 * k + 1] += phi + ((nlo < olo) ? 1ull : 0ull);
      }
    }
  };
  // Pairs (ra, rb), ra < rb, of the staged row: warps take rows ra from a
  // shared counter (long rows first), lanes take rb. A staged entry's fourth
  // word is the hub edge's bin, premultiplied by nb for the configuration
  // table. EXACT: every bin edge E_b^2 is a multiple of the bucket width, so
  // a bucket holds one bin (or 0xFF below E_0) and the bucket lookup is the
  // whole test; otherwise the squared distance is range-tested and the
  // bucket's bin is finished by one comparison with the next edge.
  const uint32_t s_hist = (uint32_t)__cvta_generic_to_shared(sm.hist);
  const uint32_t s_hacc = WEIGHTED ? (uint32_t)__cvta_generic_to_shared(sm.hacc) : 0u;
  const unsigned long long span = (unsigned long long)(e2hi - e2lo);
  // a staged entry's x displacement and tag (see the staging loop)
  auto ent_x = [](const int4& e) -> int {
    return WEIGHTED ? (int)((uint32_t)e.x << 11) >> 11 : e.x;
  };
  auto ent_tag = [](const int4& e) -> int {
    return WEIGHTED ? (int)((uint32_t)e.x >> 21) : e.w;
  };
  auto pair = [&](int xa, const int4& Da, int taga, const int4& Db, int abase, int32_t Wa) {
    const int x = ent_x(Db) - xa, y = Db.y - Da.y, z = Db.z - Da.z;
    const unsigned long long D2 =
        (unsigned long long)((long long)x * x + (long long)y * y + (long long)z * z);
    int bjk;
    if constexpr (BIN == kBinLinear) {
      // q < (m nb)^2 <= 2^18 is exact in FP32; for q in [(m b)^2, (m (b+1))^2)
      // sqrt(q) / m lies in [b, b + 1 - 1 / (2 m^2 (b + 1))], and the
      // approximate square root (relative error below 2^-22 with the
      // multiply) raised by 2^-20 lands strictly inside [b, b + 1) when
      // m nb <= 512, so truncation gives b exactly
      const unsigned long long q = D2 >> a.bk_shift;
      if (q >= (unsigned long long)a.bk_n) return;
      float r;
      asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"((float)(uint32_t)q));
      bjk = (int)(r * a.lin_c);
    } else if constexpr (BIN == kBinTable) {
      const unsigned long long q = D2 >> a.bk_shift;
      if (q >= (unsigned long long)a.bk_n) return;
      bjk = bk[q];
      if (bjk == 0xFF) return;
    } else {
      if (D2 - (unsigned long long)e2lo >= span) return;
      if (bk) {
        const int b0 = bk[D2 >> a.bk_shift];
        bjk = b0 + ((long long)D2 >= s_e2[b0 + 1] ? 1 : 0);
      } else {
        int lo = 0, hi = nb;
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (s_e2[mid] <= (long long)D2) lo = mid;
          else hi = mid;
        }
        bjk = lo;
      }
    }
    const int tagb = ent_tag(Db);
    const int cf = LUT ? (int)sm.lut[abase + tagb + bjk] : conf3_rank(taga, tagb, bjk, nb);
    record_if<WM>(s_hist, s_hacc, cf, true, Wa, WEIGHTED ? Db.w : 0);
  };
  auto pairs = [&](const int4* S, int d) {
    for (;;) {
      int ra = 0;
      if (lane == 0) ra = atomicAdd(&s_next, 1);
      ra = __shfl_sync(0xffffffffu, ra, 0);
      if (ra >= d - 1) break;
      const int4 Da = S[ra];
      const int xa = ent_x(Da), taga = ent_tag(Da);
      const int32_t Wa = WEIGHTED ? Da.w : 0;
      const int abase = LUT ? taga * nb : 0;  // b_ij nb^2
      int rb = ra + 1 + lane;
      for (; rb + 32 < d; rb += 64) {
        const int4 D0 = S[rb], D1 = S[rb + 32];
        pair(xa, Da, taga, D0, abase, Wa);
        pair(xa, Da, taga, D1, abase, Wa);
      }
      if (rb < d) pair(xa, Da, taga, S[rb], abase, Wa);
    }
  };

  for (;;) {
    if (tid == 0) {
      const int64_t q = (int64_t)atomicAdd(a.hub_counter, 1ull);
      int k = 0;
      int64_t hub;
      bool valid;
      if (BATCH) {
        valid = q < a.base[a.ncats];
        if (valid) {
          int lo = 0, hi = a.ncats;  // largest k with base[k] <= q
          while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (a.base[mid] <= q) lo = mid;
            else hi = mid;
          }
          k = lo;
        }
        hub = valid ? q - a.base[k] : 0;
      } else {
        hub = a.one.hub_begin + q;
        valid = hub < a.one.hub_end;
      }
      s_hub = valid ? hub : -1;
      s_cat = k;
      s_flush = 0;
      s_next = 0;
      if (valid) {
        const int32_t* dg = BATCH ? a.cats[k].deg : a.one.deg;
        const unsigned long long d = (unsigned long long)dg[hub];
        const unsigned long long need = d * (d - (d > 0)) / 2;  // triangles at i <= C(d,2)
        if (k != s_cur || s_pending + need > 0xFFFFFFFFull) {
          s_flush = 1;
          s_pending = need;
          s_cur = k;
        } else {
          s_pending += need;
        }
      }
    }
    __syncthreads();
    const int64_t i = s_hub;
    if (i < 0) break;
    if (s_flush) {
      flush();
      __syncthreads();
    }
    if (BATCH && s_cat != cur) {
      cur = s_cat;
      c = a.cats[cur];
    }
    const int d = c.deg[i];
    if (d < 2) {
      __syncthreads();
      continue;
    }
    const uint32_t* row = row_at(c.adj, c.ptr, i, c.adj_off, c.split, c.adj_off2);
    const int4 P = c.xyzp[i];
    const bool big = d > a.cap;
    int4* gS = reinterpret_cast<int4*>(a.gscratch + (size_t)blockIdx.x * a.gstride);
    int4* S = big ? gS : s_stage;
    for (int t = tid; t < d; t += kPThreads) {
      const uint32_t w = row[t];
      const uint32_t k = edge_id(w);
      const int4 Q = c.xyzp[k];
      const int dx = (int)min_image((int64_t)Q.x - P.x, c.box);
      const int tag = (int)edge_bin(w) * (LUT ? nb : 1);
      // weighted: the tag rides in bits 21..30 above the 21-bit x
      // displacement (|dx| < 2^19), the fourth word is W_k
      S[t] = make_int4(WEIGHTED ? (int)(((uint32_t)dx & 0x1FFFFFu) | ((uint32_t)tag << 21)) : dx,
                       (int)min_image((int64_t)Q.y - P.y, c.box),
                       (int)min_image((int64_t)Q.z - P.z, c.box),
                       WEIGHTED ? (int)c.W[k] : tag);
    }
    __syncthreads();
    if (big) pairs(gS, d);
    else pairs(s_stage, d);
    __syncthreads();
    fold_hub(WEIGHTED ? (int64_t)c.W[i] : 0);
  }
  __syncthreads();
  flush();
}

// Equilateral configurations (b, b, b) by pair geometry: a triangle is
// equilateral in this sense only when both hub edges share bin b, so the CTA
// stages N+(i) grouped by the hub edge's bin (a counting sort in shared
// memory) and tests only the pairs within a group, against the one range
// [E_b, E_b+1). Counts go to per-CTA 32-bit histograms [nb]; weighted, W_j W_k
// to the hub's 96-bit sums [nb] folded by W_i into the CTA's 128-bit sums,
// as in the other triangle kernels.
template <int WM>
__global__ void __launch_bounds__(kPThreads, 2) k_equi3p(PArgs a) {
  constexpr bool WEIGHTED = WM != kNone;
  extern __shared__ __align__(16) unsigned char smem[];
  int4* s_stage = reinterpret_cast<int4*>(smem);
  __shared__ int64_t s_e2[kMaxBins + 1];
  __shared__ int s_cnt[kMaxBins + 1], s_cur[kMaxBins + 1];
  __shared__ unsigned s_hist[kMaxBins];
  __shared__ unsigned s_hacc[WEIGHTED ? 3 * kMaxBins : 1];
  __shared__ unsigned long long s_whist[WEIGHTED ? 2 * kMaxBins : 1];
  __shared__ int64_t s_hub;
  __shared__ unsigned long long s_pending;
  __shared__ int s_flush, s_next;
  const int tid = threadIdx.x, lane = tid & 31;
  const int nb = a.nb;
  for (int b = tid; b <= nb; b += kPThreads) s_e2[b] = a.e2g[b];
  for (int b = tid; b < nb; b += kPThreads) {
    s_hist[b] = 0u;
    if (WEIGHTED) {
      s_hacc[3 * b] = s_hacc[3 * b + 1] = s_hacc[3 * b + 2] = 0u;
      s_whist[2 * b] = s_whist[2 * b + 1] = 0ull;
    }
  }
  if (tid == 0) s_pending = 0;
  __syncthreads();
  const Cat c = a.one;

  auto flush = [&]() {
    for (int b = tid; b < nb; b += kPThreads) {
      const unsigned v = s_hist[b];
      if (v) {
        atomicAdd(c.counts + b, (unsigned long long)v);
        s_hist[b] = 0u;
      }
      if (WEIGHTED) {
        const unsigned long long lo = s_whist[2 * b], hi = s_whist[2 * b + 1];
        if (lo | hi) {
          atomic_add_i192(c.wacc + 3 * b, lo, hi);
          s_whist[2 * b] = s_whist[2 * b + 1] = 0ull;
        }
      }
    }
  };

  for (;;) {
    if (tid == 0) {
      const int64_t i = c.hub_begin + (int64_t)atomicAdd(a.hub_counter, 1ull);
      s_hub = i < c.hub_end ? i : -1;
      s_flush = 0;
      s_next = 0;
      if (i < c.hub_end) {
        const unsigned long long d = (unsigned long long)c.deg[i];
        const unsigned long long need = d * (d - (d > 0)) / 2;
        if (s_pending + need > 0xFFFFFFFFull) {
          s_flush = 1;
          s_pending = need;
        } else {
          s_pending += need;
        }
      }
    }
    for (int b = tid; b <= nb; b += kPThreads) s_cnt[b] = 0;
    __syncthreads();
    const int64_t i = s_hub;
    if (i < 0) break;
    if (s_flush) {
      flush();
      __syncthreads();
    }
    const int d = c.deg[i];
    if (d < 2) {
      __syncthreads();
      continue;
    }
    const uint32_t* row = row_at(c.adj, c.ptr, i, c.adj_off, c.split, c.adj_off2);
    const int4 P = c.xyzp[i];
    int4* S = d > a.cap ? reinterpret_cast<int4*>(a.gscratch + (size_t)blockIdx.x * a.gstride)
                        : s_stage;
    uint8_t* G = reinterpret_cast<uint8_t*>(S + (d > a.cap ? d : a.cap));  // group of each entry
    // counting sort of the row by hub-edge bin
    for (int t = tid; t < d; t += kPThreads) atomicAdd(&s_cnt[edge_bin(row[t]) + 1], 1);
    __syncthreads();
    if (tid == 0) {
      for (int b = 1; b <= nb; ++b) s_cnt[b] += s_cnt[b - 1];
      for (int b = 0; b < nb; ++b) s_cur[b] = s_cnt[b];
    }
    __syncthreads();
    for (int t = tid; t < d; t += kPThreads) {
      const uint32_t w = row[t];
      const uint32_t k = edge_id(w);
      const int4 Q = c.xyzp[k];
      const int pos = atomicAdd(&s_cur[edge_bin(w)], 1);
      G[pos] = (uint8_t)edge_bin(w);
      S[pos] = make_int4((int)min_image((int64_t)Q.x - P.x, c.box),
                         (int)min_image((int64_t)Q.y - P.y, c.box),
                         (int)min_image((int64_t)Q.z - P.z, c.box),
                         WEIGHTED ? (int)c.W[k] : (int)edge_bin(w));
    }
    __syncthreads();
    // warps take four rows ra0..ra0+3 at a time; the pairs (ra, rb) with rb
    // later in ra's group are spread over the lanes as one list
    for (;;) {
      int ra0 = 0;
      if (lane == 0) ra0 = atomicAdd(&s_next, 4);
      ra0 = __shfl_sync(0xffffffffu, ra0, 0);
      if (ra0 >= d - 1) break;
      int nk = 0;  // partners of row ra0 + lane (lanes 0..3)
      if (lane < 4 && ra0 + lane < d - 1) nk = s_cnt[G[ra0 + lane] + 1] - (ra0 + lane) - 1;
      int pre = nk;
      for (int o = 1; o < 4; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, pre, o);
        if (lane >= o) pre += v;
      }
      const int p0 = __shfl_sync(0xffffffffu, pre, 0), p1 = __shfl_sync(0xffffffffu, pre, 1),
                p2 = __shfl_sync(0xffffffffu, pre, 2), T = __shfl_sync(0xffffffffu, pre, 3);
      for (int t = lane; t < T; t += 32) {
        const int k = (t >= p0 ? 1 : 0) + (t >= p1 ? 1 : 0) + (t >= p2 ? 1 : 0);
        const int base = k == 0 ? 0 : (k == 1 ? p0 : (k == 2 ? p1 : p2));
        const int ra = ra0 + k, rb = ra + 1 + (t - base);
        const int b = G[ra];
        const int4 Da = S[ra], Db = S[rb];
        const int64_t x = (int64_t)Db.x - Da.x, y = (int64_t)Db.y - Da.y,
                      z = (int64_t)Db.z - Da.z;
        const int64_t D2 = x * x + y * y + z * z;
        if (D2 < s_e2[b] || D2 >= s_e2[b + 1]) continue;
        atomicAdd(&s_hist[b], 1u);
        if constexpr (WEIGHTED) {
          const long long xw = (long long)Da.w * Db.w;  // |.| < 2^60
          const uint32_t x0 = (uint32_t)xw, x1 = (uint32_t)((unsigned long long)xw >> 32);
          const uint32_t o0 = atomicAdd(&s_hacc[3 * b], x0);
          const uint32_t a1 = x1 + ((o0 + x0 < o0) ? 1u : 0u);
          uint32_t a2 = (xw < 0 ? 0xFFFFFFFFu : 0u) + ((a1 < x1) ? 1u : 0u);
          if (a1) {
            const uint32_t o1 = atomicAdd(&s_hacc[3 * b + 1], a1);
            a2 += (o1 + a1 < o1) ? 1u : 0u;
          }
          if (a2) atomicAdd(&s_hacc[3 * b + 2], a2);
        }
      }
    }
    __syncthreads();
    if constexpr (WEIGHTED) {
      // the hub's 96-bit sums times W_i into the CTA's 128-bit sums
      const int64_t Wi = c.W[i];
      for (int b = tid; b < nb; b += kPThreads) {
        const uint32_t l = s_hacc[3 * b], m = s_hacc[3 * b + 1], h = s_hacc[3 * b + 2];
        if (!(l | m | h)) continue;
        s_hacc[3 * b] = s_hacc[3 * b + 1] = s_hacc[3 * b + 2] = 0u;
        const unsigned long long ml = ((unsigned long long)m << 32) | l;
        const unsigned long long uw = (unsigned long long)Wi;
        const unsigned long long plo = ml * uw;
        unsigned long long phi = __umul64hi(ml, uw) - (Wi < 0 ? ml : 0ull);
        phi += (unsigned long long)((long long)(int32_t)h * Wi);
        const unsigned long long olo = s_whist[2 * b];
        const unsigned long long nlo = olo + plo;
        s_whist[2 * b] = nlo;
        s_whist[2 * b + 1] += phi + ((nlo < olo) ? 1ull : 0ull);
      }
    }
  }
  __syncthreads();
  flush();
}

template <bool BATCH>
void (*pick_count3p(int wm, bool nonneg, bool lut, int bin))(PArgs) {
#define GS_P2(W, L)                                                        \
  (bin == kBinLinear  ? k_count3p<W, BATCH, L, kBinLinear>                 \
   : bin == kBinTable ? k_count3p<W, BATCH, L, kBinTable>                  \
                      : k_count3p<W, BATCH, L, kBinSearch>)
#define GS_P(W) (lut ? GS_P2(W, true) : GS_P2(W, false))
  if (wm == kNone) return GS_P(kNone);
  return nonneg ? GS_P(kExactPos) : GS_P(kExact);
#undef GS_P
#undef GS_P2
}

// Shared-memory layout of k_count3: the direct-address table takes what the
// staging buffer, configuration table and histograms leave.
struct Count3Launch {
  size_t smem = 0;
  int span_cap = 0;
  int stage_words = 0;
  bool smem_hist = true;
  bool lut = false;  // the configuration table is staged
};

// Hubs with more than kMaxSmemHistDeg neighbours could overflow the 32-bit
// shared counters within one hub; graphs with such rows count straight into
// the global histograms.
constexpr int kMaxSmemHistDeg = 65535;

Count3Launch count3_launch(int nb, int nconf, int wmode, bool use_lut, bool compact,
                           bool ring, int max_deg) {
  const bool weighted = wmode != kNone;
  // weighted launches stage rows and weights of up to 2048 neighbours
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  auto pad16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
  const size_t nb3 = (size_t)nb * nb * nb;
  const size_t lut = (use_lut && nb3 <= (size_t)kLutMax) ? pad16(nb3 * 2) : 0;
  // counts, then (weighted) the CTA's 128-bit sums and the hub's 96-bit sums
  size_t hist = pad16((size_t)nconf * 4) + (wmode >= kExact ? pad16((size_t)nconf * 28) : 0);
  Count3Launch L;
  L.lut = lut != 0;
  const size_t avail = (size_t)optin - 2048;  // static shared memory and slack
  const size_t stage_words = weighted ? 2048 : kStageCap;
  const size_t queue = (weighted && compact) ? (size_t)kWarps * 128 * 4 : 0;
  const size_t ringb = ring ? (size_t)kWarps * kRing * (128 * 4 + 4) : 0;
  const size_t fixed = stage_words * (weighted ? 12 : 4) + queue + ringb + lut;
  L.smem_hist = fixed + hist + 32 * 1024 <= avail && max_deg <= kMaxSmemHistDeg;
  if (!L.smem_hist) hist = 0;
  L.span_cap = (int)((avail - fixed - hist) & ~(size_t)15);
  L.stage_words = (int)stage_words;
  L.smem = (size_t)L.span_cap + fixed + hist;
  return L;
}

// Launch plan of the pair kernel: shared-memory layout sized for two CTAs
// per SM when it fits (one otherwise), squared-distance buckets, and the
// global staging for hubs above the shared capacity.
struct PairLaunch {
  size_t smem = 0;
  int cap = 0;
  int per_sm = 0;
  bool lut = false;
  int bin = kBinSearch;
  int bk_shift = 0, bk_n = 0;  // kBinLinear: q = D2 >> bk_shift, edges iff q < bk_n
  float lin_c = 0.0f;
};

PairLaunch pair_launch(int nb, int nconf, bool weighted, bool use_lut,
                       const std::vector<int64_t>& edges) {
  PairLaunch L;
  int dev = 0, optin = 0, per_sm_bytes = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&per_sm_bytes, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  auto pad16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
  // Exact buckets when every squared edge is a multiple of a power of two
  // 2^sx that leaves at most kPBucketExactMax buckets below E_nb^2 (edges
  // on a coarse lattice, e.g. E_b = 2048 b); otherwise buckets no wider
  // than the narrowest bin in squared distance, finished by a comparison.
  const int64_t top = edges[nb] * edges[nb];
  int sx = 62;
  for (int b = 0; b <= nb; ++b) {
    const int64_t e2 = edges[b] * edges[b];
    if (e2) sx = std::min(sx, __builtin_ctzll((unsigned long long)e2));
  }
  const int64_t nbx = ((top - 1) >> sx) + 1;
  // linear bins from zero: E_b = b E_1 with E_1 = m 2^t, m odd, m nb <= 512
  bool linear = edges[0] == 0 && edges[1] > 0;
  for (int b = 2; b <= nb && linear; ++b) linear = edges[b] == b * edges[1];
  int t = 0;
  int64_t m = linear ? edges[1] : 0;
  while (linear && m % 2 == 0) {
    m /= 2;
    ++t;
  }
  if (linear && m * nb <= 512) {
    L.bin = kBinLinear;
    L.bk_shift = 2 * t;
    L.bk_n = (int)(m * m * nb * nb);  // (E_nb / 2^t)^2
    L.lin_c = (float)((1.0 / (double)m) * (1.0 + std::ldexp(1.0, -20)));
  } else if (nbx <= kPBucketExactMax && nb < 255) {
    L.bin = kBinTable;
    L.bk_shift = sx;
    L.bk_n = (int)nbx;
  } else {
    int64_t gap = INT64_MAX;
    for (int b = 0; b < nb; ++b)
      gap = std::min(gap, edges[b + 1] * edges[b + 1] - edges[b] * edges[b]);
    int sh = 0;
    while (sh < 62 && (int64_t(1) << (sh + 1)) <= gap) ++sh;
    const int64_t nbk = ((top - 1) >> sh) + 1;
    if (gap >= 1 && nbk <= kPBucketMax) {
      L.bk_shift = sh;
      L.bk_n = (int)nbk;
    }
  }
  const size_t nb3 = (size_t)nb * nb * nb;
  L.lut = use_lut && nb3 <= (size_t)kLutMax;
  const size_t fixed = pad16((size_t)(nb + 1) * 8) + (L.lut ? pad16(nb3 * 2) : 0) +
                       pad16((size_t)nconf * 4) + (weighted ? (size_t)nconf * 28 : 0) +
                       (L.bin == kBinLinear ? 0 : pad16((size_t)L.bk_n));
  const size_t per = 16;  // one int4 per staged neighbour
  const size_t static_bytes = 256;  // the kernel's own __shared__ variables and slack
  for (int ctas = 2; ctas >= 1; --ctas) {
    const size_t budget =
        std::min((size_t)optin, (size_t)per_sm_bytes / ctas - 1024) - static_bytes;
    if (budget <= fixed) continue;
    int cap = (int)std::min<size_t>(4096, (budget - fixed) / per) & ~31;
    if (cap < 256 && ctas == 2) continue;
    if (cap < 32) continue;
    L.cap = cap;
    L.smem = (size_t)cap * per + fixed;
    L.per_sm = ctas;
    return L;
  }
  return L;  // cap 0: the configuration tables leave no room (walk kernel instead)
}

}  // namespace

// An exact 192-bit two's-complement sum times 2^-scale, rounded to the
// nearest double with ties to even. The magnitude is first rounded to odd
// at 64 significant bits (the dropped bits only force the lowest kept bit
// to 1); the hardware's round-to-nearest conversion of that 64-bit integer
// then gives the correctly rounded double, because rounding to odd with at
// least two bits more than the target precision (64 >= 53 + 2) cannot make
// the second rounding go wrong (S. Boldo, G. Melquiond, "Emulation of FMA
// and correctly rounded sums: proved algorithms using rounding to odd",
// IEEE Trans. Computers 57(4), 2008). The final power-of-two scaling is
// exact: FP32 weights keep every scaled sum far above 2^-1022.
__global__ void k_i192_to_double(const unsigned long long* acc, int64_t n, int scale,
                                 double* out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long a0 = acc[3 * k], a1 = acc[3 * k + 1], a2 = acc[3 * k + 2];
    const bool neg = (long long)a2 < 0;
    if (neg) {  // |value| = ~value + 1 across the three limbs
      a0 = ~a0;
      a1 = ~a1;
      a2 = ~a2;
      if (++a0 == 0ull && ++a1 == 0ull) ++a2;
    }
    unsigned long long top, lost;  // the 64-bit window and the bits below it
    int below;                     // how many bits lie below the window
    if (a2) {
      const int z = __clzll((long long)a2);
      top = z ? (a2 << z) | (a1 >> (64 - z)) : a2;
      lost = (z ? a1 << z : a1) | a0;
      below = 128 - z;
    } else if (a1) {
      const int z = __clzll((long long)a1);
      top = z ? (a1 << z) | (a0 >> (64 - z)) : a1;
      lost = z ? a0 << z : a0;
      below = 64 - z;
    } else {
      top = a0;
      lost = 0ull;
      below = 0;
    }
    top |= (lost != 0ull) ? 1ull : 0ull;  // round to odd
    const double v = scalbn(__ull2double_rn(top), below - scale);
    out[k] = neg ? -v : v;
  }
}

__global__ void k_u64_to_double(const unsigned long long* c, int64_t n, double* out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    out[k] = (double)c[k];
}

int resolve_variant(const Graph& g, int wmode, int variant);

int count3_device(const Graph& g, const FixedW* fw, uint64_t* d_counts, double* d_wsum,
                  const Opts& o_in, Scratch& sc, bool equi, unsigned long long* wacc_out) {
  Opts o = o_in;
  const bool weighted = fw && (d_wsum || wacc_out);
  o.variant = equi ? std::max(o.variant, 0) : resolve_variant(g, weighted ? 2 : 0, o.variant);
  cudaStream_t s = o.stream;
  // the equilateral configurations (b, b, b) are indexed by b
  const int nconf = equi ? g.nb : (int)num_conf3(g.nb);
  Args a;
  a.one.ptr = g.d_ptr;
  a.one.deg = g.d_deg;
  a.one.adj = nullptr;
  a.one.adj_off = 0;
  a.one.split = g.n;
  a.one.adj_off2 = 0;
  a.cats = nullptr;
  a.base = nullptr;
  a.ncats = 0;
  a.nb = g.nb;
  a.nconf = nconf;
  // variant 1: every hub through the hash path in 64-word segments;
  // variant 2: the table path reading hub rows from global memory
  a.seg_cap = (o.variant & 1) ? 64 : kSegCap;
  a.force_hash = (o.variant & 1) ? 1 : 0;
  a.stage_cap = (o.variant & 2) ? 0 : kStageCap;
  a.one.counts = reinterpret_cast<unsigned long long*>(d_counts);
  a.one.W = fw ? fw->d_W : nullptr;
  const int wm = weighted ? kExact : kNone;
  a.one.wacc = wm == kExact ? (wacc_out ? wacc_out : sc.alloc<unsigned long long>(3 * (size_t)nconf))
                            : nullptr;
  a.hub_counter = sc.alloc<unsigned long long>(1);
  a.err = sc.alloc<int>(1);
  if (!a.hub_counter || !a.err || (wm == kExact && !a.one.wacc)) return GS_ENOMEM;
  cudaMemsetAsync(d_counts, 0, sizeof(uint64_t) * nconf, s);
  if (wm == kExact) cudaMemsetAsync(a.one.wacc, 0, sizeof(unsigned long long) * 3 * nconf, s);
  cudaMemsetAsync(a.err, 0, sizeof(int), s);
  if (g.n == 0) {
    if (d_wsum) cudaMemsetAsync(d_wsum, 0, sizeof(double) * nconf, s);
    return cuda_status(cudaGetLastError());
  }

  const bool use_lut = !equi && !(o.variant & 4);
  a.one.xyzp = g.d_xyzp;
  a.one.box = g.box_u;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  KernelTimer timer(o.kernel_ms);
  int st = GS_OK;
  // The pair kernel is the default. Launch bits of the walk's own paths
  // (1, 2, 8, 16, 32, 64, 512), the equilateral configurations and rows of
  // more than 65,535 neighbours (whose triangles could overflow the 32-bit
  // shared counters within one hub) take the merge-walk kernel.
  const bool pair_ok = !equi && (o.variant & ~4) == 0 && g.max_deg <= kMaxSmemHistDeg;
  const PairLaunch PL = pair_ok ? pair_launch(g.nb, nconf, wm != kNone, use_lut, g.edges)
                                : PairLaunch{};
  // equilateral configurations: pair geometry within hub-edge bin groups
  // (variant bit 512 keeps the walk's EQUI instantiation)
  const bool equi_pair = equi && !(o.variant & 512) && g.max_deg <= kMaxSmemHistDeg;
  if (equi_pair) {
    PArgs pa;
    pa.one = a.one;
    pa.cats = nullptr;
    pa.base = nullptr;
    pa.ncats = 0;
    pa.nb = g.nb;
    pa.nconf = nconf;
    pa.use_lut = 0;
    pa.bk_shift = pa.bk_n = 0;
    pa.lin_c = 0.0f;
    pa.e2g = g.d_edges2;
    pa.hub_counter = a.hub_counter;
    int per_sm_bytes = 0;
    cudaDeviceGetAttribute(&per_sm_bytes, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    // two CTAs per SM: the staging buffer takes what the static arrays leave
    const size_t budget = (size_t)per_sm_bytes / 2 - 1024 - 16 * 1024;
    pa.cap = (int)std::min<size_t>(4096, budget / 17) & ~31;
    const size_t smem = (size_t)pa.cap * 17;
    void (*kern)(PArgs) = wm == kNone ? k_equi3p<kNone> : k_equi3p<kExact>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPThreads, smem);
    const int grid = std::max(1, per_sm) * sms;
    pa.gscratch = nullptr;
    pa.gstride = 0;
    if (g.max_deg > pa.cap) {
      pa.gstride = ((size_t)g.max_deg * 17 + 255) & ~(size_t)255;
      pa.gscratch = sc.alloc<unsigned char>(pa.gstride * grid);
      if (!pa.gscratch) return GS_ENOMEM;
    }
    timer.start(s);
    st = for_each_window(g, o, sc, [&](const WinView& v) -> int {
      pa.one.adj = v.adj;
      pa.one.adj_off = v.off1;
      pa.one.split = v.split;
      pa.one.adj_off2 = v.off2;
      pa.one.hub_begin = v.h0;
      pa.one.hub_end = v.h1;
      cudaMemsetAsync(pa.hub_counter, 0, sizeof(unsigned long long), s);
      { kern<<<grid, kPThreads, smem, s>>>(pa); note_launch(); }
      return cuda_status(cudaGetLastError());
    });
    timer.stop(s);
  } else if (PL.cap > 0) {
    PArgs pa;
    pa.one = a.one;
    pa.cats = nullptr;
    pa.base = nullptr;
    pa.ncats = 0;
    pa.nb = g.nb;
    pa.nconf = nconf;
    pa.cap = PL.cap;
    pa.use_lut = PL.lut ? 1 : 0;
    pa.bk_shift = PL.bk_shift;
    pa.bk_n = PL.bk_n;
    pa.e2g = g.d_edges2;
    pa.hub_counter = a.hub_counter;
    pa.lin_c = PL.lin_c;
    void (*kern)(PArgs) =
        pick_count3p<false>(wm, fw && fw->nonneg, PL.lut, PL.bin);
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PL.smem);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPThreads, PL.smem);
    const int grid = std::max(1, per_sm) * sms;
    pa.gscratch = nullptr;
    pa.gstride = 0;
    if (g.max_deg > PL.cap) {
      pa.gstride = ((size_t)g.max_deg * 16 + 255) & ~(size_t)255;
      pa.gscratch = sc.alloc<unsigned char>(pa.gstride * grid);
      if (!pa.gscratch) return GS_ENOMEM;
    }
    timer.start(s);
    st = for_each_window(g, o, sc, [&](const WinView& v) -> int {
      pa.one.adj = v.adj;
      pa.one.adj_off = v.off1;
      pa.one.split = v.split;
      pa.one.adj_off2 = v.off2;
      pa.one.hub_begin = v.h0;
      pa.one.hub_end = v.h1;
      cudaMemsetAsync(pa.hub_counter, 0, sizeof(unsigned long long), s);
      { kern<<<grid, kPThreads, PL.smem, s>>>(pa); note_launch(); }
      return cuda_status(cudaGetLastError());
    });
    timer.stop(s);
  } else {
  const Count3Launch L =
      count3_launch(g.nb, nconf, wm, use_lut, (o.variant & 32) != 0, (o.variant & 64) != 0,
                    g.max_deg);
  a.span_cap = (o.variant & 8) ? 2048 : L.span_cap;
  a.stage_alloc = L.stage_words;
  a.use_lut = use_lut ? 1 : 0;
  a.compact = (o.variant & 32) ? 1 : 0;
  a.ring = (o.variant & 64) ? 1 : 0;
  a.first_wait_limit = (o.variant & 16) ? 0u : kWaitLimit;
  a.stage_cap = std::min(a.stage_cap, L.stage_words);
  const bool smem_hist = L.smem_hist;
  const size_t smem = L.smem;
  void (*kern)(Args);
  kern = equi ? pick_equi3(wm, fw && fw->nonneg, smem_hist)
              : pick_count3<false>(wm, fw && fw->nonneg, smem_hist, L.lut);
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
  const int grid = std::max(1, per_sm) * sms;
  timer.start(s);
  st = for_each_window(g, o, sc, [&](const WinView& v) -> int {
    a.one.adj = v.adj;
    a.one.adj_off = v.off1;
    a.one.split = v.split;
    a.one.adj_off2 = v.off2;
    a.one.hub_begin = v.h0;
    a.one.hub_end = v.h1;
    cudaMemsetAsync(a.hub_counter, 0, sizeof(unsigned long long), s);
    { kern<<<grid, kThreads, smem, s>>>(a); note_launch(); }
    return cuda_status(cudaGetLastError());
  });
  timer.stop(s);
  }
  if (st) return st;
  cudaError_t e;
  if (d_wsum) {
    if (wm == kExact)
      { k_i192_to_double<<<(nconf + 255) / 256, 256, 0, s>>>(a.one.wacc, nconf, 3 * fw->scale, d_wsum); note_launch(); }
    else if (wm == kNone)
      { k_u64_to_double<<<(nconf + 255) / 256, 256, 0, s>>>(a.one.counts, nconf, d_wsum); note_launch(); }
  }
  int herr = 0;
  cudaMemcpyAsync(&herr, a.err, sizeof(int), cudaMemcpyDeviceToHost, s);
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e);
  timer.publish();
  return herr ? GS_ETIMEOUT : GS_OK;
}

int count3_batch_device(const Graph* const* gr, int ng, const FixedW* fws, uint64_t* const* d_counts,
                        double* const* d_wsum, const Opts& o_in, Scratch& sc) {
  Opts o = o_in;
  o.variant = resolve_variant(*gr[0], (fws && d_wsum) ? 2 : 0, o.variant);
  cudaStream_t s = o.stream;
  const int nb = gr[0]->nb;
  const int nconf = (int)num_conf3(nb);
  const int wm = (fws && d_wsum) ? kExact : kNone;
  std::vector<Cat> cats(ng);
  std::vector<int64_t> base(ng + 1, 0);
  unsigned long long* wacc =
      wm == kExact ? sc.alloc<unsigned long long>(3 * (size_t)nconf * ng) : nullptr;
  if (wm == kExact && !wacc) return GS_ENOMEM;
  for (int k = 0; k < ng; ++k) {
    const Graph& g = *gr[k];
    Cat& c = cats[k];
    c.ptr = g.d_ptr;
    c.deg = g.d_deg;
    c.adj = g.d_adj;
    c.adj_off = 0;
    c.split = g.n;
    c.adj_off2 = 0;
    c.W = fws ? fws[k].d_W : nullptr;
    c.counts = reinterpret_cast<unsigned long long*>(d_counts[k]);
    c.wacc = wm == kExact ? wacc + 3 * (size_t)nconf * k : nullptr;
    c.hub_begin = 0;
    c.hub_end = g.n;
    c.xyzp = g.d_xyzp;
    c.box = g.box_u;
    base[k + 1] = base[k] + g.n;
    cudaMemsetAsync(d_counts[k], 0, sizeof(uint64_t) * nconf, s);
  }
  if (wm == kExact) cudaMemsetAsync(wacc, 0, sizeof(unsigned long long) * 3 * nconf * ng, s);
  Cat* d_cats = sc.alloc<Cat>(ng);
  int64_t* d_base = sc.alloc<int64_t>(ng + 1);
  Args a;
  a.one = cats[0];
  a.cats = d_cats;
  a.base = d_base;
  a.ncats = ng;
  a.nb = nb;
  a.nconf = nconf;
  a.seg_cap = (o.variant & 1) ? 64 : kSegCap;
  a.force_hash = (o.variant & 1) ? 1 : 0;
  a.stage_cap = (o.variant & 2) ? 0 : kStageCap;
  a.hub_counter = sc.alloc<unsigned long long>(1);
  a.err = sc.alloc<int>(1);
  if (!d_cats || !d_base || !a.hub_counter || !a.err) return GS_ENOMEM;
  cudaMemcpyAsync(d_cats, cats.data(), sizeof(Cat) * ng, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(d_base, base.data(), sizeof(int64_t) * (ng + 1), cudaMemcpyHostToDevice, s);
  cudaMemsetAsync(a.hub_counter, 0, sizeof(unsigned long long), s);
  cudaMemsetAsync(a.err, 0, sizeof(int), s);
  int max_deg = 0;
  for (int k = 0; k < ng; ++k) max_deg = std::max(max_deg, gr[k]->max_deg);
  bool nonneg = true;
  for (int k = 0; k < ng && fws; ++k) nonneg = nonneg && fws[k].nonneg;
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  KernelTimer timer(o.kernel_ms);
  // the pair kernel when the catalogues share their bin edges (one bucket
  // table serves them all), else the merge-walk kernel
  bool same_edges = true;
  for (int k = 1; k < ng; ++k) same_edges = same_edges && gr[k]->edges == gr[0]->edges;
  const bool pair_ok = same_edges && (o.variant & ~4) == 0 && max_deg <= kMaxSmemHistDeg;
  const PairLaunch PL = pair_ok ? pair_launch(nb, nconf, wm != kNone, !(o.variant & 4),
                                              gr[0]->edges)
                                : PairLaunch{};
  if (PL.cap > 0) {
    PArgs pa;
    pa.one = cats[0];
    pa.cats = d_cats;
    pa.base = d_base;
    pa.ncats = ng;
    pa.nb = nb;
    pa.nconf = nconf;
    pa.cap = PL.cap;
    pa.use_lut = PL.lut ? 1 : 0;
    pa.bk_shift = PL.bk_shift;
    pa.bk_n = PL.bk_n;
    pa.e2g = gr[0]->d_edges2;
    pa.hub_counter = a.hub_counter;
    pa.lin_c = PL.lin_c;
    void (*kern)(PArgs) =
        pick_count3p<true>(wm, nonneg, PL.lut, PL.bin);
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PL.smem);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPThreads, PL.smem);
    const int grid = std::max(1, per_sm) * sms;
    pa.gscratch = nullptr;
    pa.gstride = 0;
    if (max_deg > PL.cap) {
      pa.gstride = ((size_t)max_deg * 16 + 255) & ~(size_t)255;
      pa.gscratch = sc.alloc<unsigned char>(pa.gstride * grid);
      if (!pa.gscratch) return GS_ENOMEM;
    }
    timer.start(s);
    if (base[ng] > 0) { kern<<<grid, kPThreads, PL.smem, s>>>(pa); note_launch(); }
    timer.stop(s);
  } else {
  const Count3Launch L =
      count3_launch(nb, nconf, wm, !(o.variant & 4), (o.variant & 32) != 0, (o.variant & 64) != 0,
                    max_deg);
  a.span_cap = (o.variant & 8) ? 2048 : L.span_cap;
  a.stage_alloc = L.stage_words;
  a.use_lut = (o.variant & 4) ? 0 : 1;
  a.compact = (o.variant & 32) ? 1 : 0;
  a.ring = (o.variant & 64) ? 1 : 0;
  a.first_wait_limit = (o.variant & 16) ? 0u : kWaitLimit;
  a.stage_cap = std::min(a.stage_cap, L.stage_words);
  const bool smem_hist = L.smem_hist;
  const size_t smem = L.smem;
  void (*kern)(Args);
  kern = pick_count3<true>(wm, nonneg, smem_hist, L.lut);
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
  timer.start(s);
  if (base[ng] > 0) { kern<<<std::max(1, per_sm) * sms, kThreads, smem, s>>>(a); note_launch(); }
  timer.stop(s);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e);
  for (int k = 0; k < ng; ++k) {
    if (!d_wsum || !d_wsum[k]) continue;
    if (wm == kExact)
      { k_i192_to_double<<<(nconf + 255) / 256, 256, 0, s>>>(wacc + 3 * (size_t)nconf * k, nconf,
                                                           3 * fws[k].scale, d_wsum[k]); note_launch(); }
    else if (wm == kNone)
      { k_u64_to_double<<<(nconf + 255) / 256, 256, 0, s>>>(
          reinterpret_cast<const unsigned long long*>(d_counts[k]), nconf, d_wsum[k]); note_launch(); }
  }
  int herr = 0;
  cudaMemcpyAsync(&herr, a.err, sizeof(int), cudaMemcpyDeviceToHost, s);
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e);
  timer.publish();
  return herr ? GS_ETIMEOUT : GS_OK;
}

}  // namespace gs

// ----------------------------------------------------------------------------
// Triangle counts without any memory allocation.
//
// Some callers cannot let a library allocate device memory during a call:
// code that runs under a fixed memory plan (a serving process that has
// handed all of HBM to its own pool, so any further cudaMalloc fails), and
// real-time loops that must not hit the allocator's locks or its implicit
// device synchronisation.
// For them gs_count_3pcf_noalloc counts the triangles of a resident graph
// using only a fixed scratch array that lives in this library's device
// image for as long as the library stays loaded (every GPU that loads the
// library holds it). The array holds the kernel's hub counter and error
// flag and, when the caller's output is host memory, the counts on their
// way back, so it limits nb to kNoAllocMaxBins (C(37,3) = 7770 bins).
//
// All calls share the one array: calls whose device work overlaps (calls on
// different streams, or from several host threads, before the earlier ones
// finished) race on it and give wrong results. Every call clears what must
// start at zero before its kernel runs.
namespace gs {
namespace {
constexpr int kNoAllocMaxBins = 35;
constexpr size_t kNoAllocScratchBytes = 64 * 1024;
constexpr size_t kNoAllocCountsOffset = 256;  // counter and error flag first
constexpr size_t conf3_of(size_t nb) { return (nb + 2) * (nb + 1) * nb / 6; }
// the counts of the largest bin count must fit behind the counter and flag
static_assert(kNoAllocCountsOffset + 8 * conf3_of(kNoAllocMaxBins) <= kNoAllocScratchBytes,
              "no-allocation scratch too small for kNoAllocMaxBins");
static_assert(kNoAllocCountsOffset + 8 * conf3_of(kNoAllocMaxBins + 1) > kNoAllocScratchBytes,
              "kNoAllocMaxBins is below what the scratch holds");
}  // namespace
}  // namespace gs

static __device__ __align__(256) unsigned char g_noalloc_scratch[gs::kNoAllocScratchBytes];

namespace gs {
namespace {
// Device address of g_noalloc_scratch per device. In host code the array's
// name is only a host-side stand-in, so the address is looked up once per
// device, with that device current, and passed to the kernel.
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kNoAllocMaxDevices] = {nullptr};

int noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e);
  if (dev < 0 || dev >= kNoAllocMaxDevices) return GS_ERANGE;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return e != cudaSuccess ? cuda_status(e) : GS_ECUDA;
    }
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return GS_OK;
}
}  // namespace
}  // namespace gs

extern "C" int gs_count_3pcf_noalloc(const gs_graph* G, uint64_t* counts,
                                     const gs_options* options) {
  using namespace gs;
  if (!G || !counts) return GS_EINVAL;
  const Graph& g = G->g;
  if (!g.d_adj) return GS_EINVAL;  // out-of-core graphs need window buffers
  if (g.nb > kNoAllocMaxBins) return GS_ERANGE;
  Opts o = read_opts(options);
  // variant -1 means the tuned choice, as for gs_count_3pcf (a table lookup,
  // no allocation)
  o.variant = resolve_variant(g, 0, o.variant);
  cudaStream_t s = o.stream;
  const int nconf = (int)num_conf3(g.nb);
  void* scratch = nullptr;
  int st = noalloc_scratch(&scratch);
  if (st) return st;
  unsigned char* base = static_cast<unsigned char*>(scratch);
  unsigned long long* counter = reinterpret_cast<unsigned long long*>(base);
  int* err = reinterpret_cast<int*>(base + 8);
  const bool dev_out = is_device_ptr(counts);
  uint64_t* dc = dev_out ? counts : reinterpret_cast<uint64_t*>(base + kNoAllocCountsOffset);
  cudaError_t e = cudaMemsetAsync(base, 0, 16, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(dc, 0, sizeof(uint64_t) * nconf, s);
  if (e != cudaSuccess) return cuda_status(e);
  if (g.n > 0) {
    Args a;
    a.one.ptr = g.d_ptr;
    a.one.deg = g.d_deg;
    a.one.adj = g.d_adj;
    a.one.adj_off = 0;
    a.one.split = g.n;
    a.one.adj_off2 = 0;
    a.one.W = nullptr;
    a.one.counts = reinterpret_cast<unsigned long long*>(dc);
    a.one.wacc = nullptr;
    a.one.hub_begin = 0;
    a.one.hub_end = g.n;
    a.one.xyzp = g.d_xyzp;
    a.one.box = g.box_u;
    a.cats = nullptr;
    a.base = nullptr;
    a.ncats = 0;
    a.nb = g.nb;
    a.nconf = nconf;
    a.seg_cap = (o.variant & 1) ? 64 : kSegCap;
    a.force_hash = (o.variant & 1) ? 1 : 0;
    a.stage_cap = (o.variant & 2) ? 0 : kStageCap;
    a.hub_counter = counter;
    a.err = err;
    const Count3Launch L =
        count3_launch(g.nb, nconf, kNone, !(o.variant & 4), false, false, g.max_deg);
    a.span_cap = (o.variant & 8) ? 2048 : L.span_cap;
    a.stage_alloc = L.stage_words;
    a.use_lut = (o.variant & 4) ? 0 : 1;
    a.compact = 0;
    a.ring = 0;
    a.first_wait_limit = (o.variant & 16) ? 0u : kWaitLimit;
    a.stage_cap = std::min(a.stage_cap, L.stage_words);
    void (*kern)(Args) = pick_count3<false>(kNone, true, L.smem_hist, L.lut);
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
    int per_sm = 0, sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, L.smem);
    { kern<<<std::max(1, per_sm) * sms, kThreads, L.smem, s>>>(a); note_launch(); }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e);
  }
  if (!dev_out) {
    e = cudaMemcpyAsync(counts, dc, sizeof(uint64_t) * nconf, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_status(e);
  }
  int herr = 0;
  e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e);
  return herr ? GS_ETIMEOUT : GS_OK;
}

// ----------------------------------------------------------------------------
// Recorded batched launches. A plan uploads the catalogue descriptors once,
// records the launch sequence of one batched count (clearing the outputs,
// the persistent kernel) into a CUDA graph, and replays it on request:
// repeated queries on resident catalogues then cost one graph launch, with
// no allocation and no host synchronisation per replay.
struct gs_plan {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  void* d_cats = nullptr;
  int64_t* d_base = nullptr;
  unsigned long long* counter = nullptr;
  int* err = nullptr;
};

extern "C" int gs_plan_3pcf_batch(const gs_graph* const* graphs, int32_t n_graphs,
                                  uint64_t* const* counts, const gs_options* options,
                                  gs_plan** out) {
  using namespace gs;
  if (!graphs || !counts || !out || n_graphs < 1) return GS_EINVAL;
  *out = nullptr;
  const int nb = graphs[0] ? graphs[0]->g.nb : 0;
  for (int k = 0; k < n_graphs; ++k) {
    if (!graphs[k] || !counts[k] || graphs[k]->g.nb != nb || !graphs[k]->g.d_adj) return GS_EINVAL;
    if (!is_device_ptr(counts[k])) return GS_EINVAL;
  }
  const Opts o = read_opts(options);
  const int nconf = (int)num_conf3(nb);
  gs_plan* P = new (std::nothrow) gs_plan();
  if (!P) return GS_ENOMEM;
  std::vector<Cat> cats(n_graphs);
  std::vector<int64_t> base(n_graphs + 1, 0);
  for (int k = 0; k < n_graphs; ++k) {
    const Graph& g = graphs[k]->g;
    Cat& c = cats[k];
    c.ptr = g.d_ptr;
    c.deg = g.d_deg;
    c.adj = g.d_adj;
    c.adj_off = 0;
    c.split = g.n;
    c.adj_off2 = 0;
    c.W = nullptr;
    c.counts = reinterpret_cast<unsigned long long*>(counts[k]);
    c.wacc = nullptr;
    c.hub_begin = 0;
    c.hub_end = g.n;
    c.xyzp = g.d_xyzp;
    c.box = g.box_u;
    base[k + 1] = base[k] + g.n;
  }
  cudaError_t e = cudaMalloc(&P->d_cats, sizeof(Cat) * n_graphs);
  if (e == cudaSuccess) e = cudaMalloc(&P->d_base, sizeof(int64_t) * (n_graphs + 1));
  if (e == cudaSuccess) e = cudaMalloc(&P->counter, sizeof(unsigned long long) + sizeof(int) + 8);
  if (e == cudaSuccess) {
    P->err = reinterpret_cast<int*>(P->counter + 1);
    e = cudaMemcpy(P->d_cats, cats.data(), sizeof(Cat) * n_graphs, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess)
    e = cudaMemcpy(P->d_base, base.data(), sizeof(int64_t) * (n_graphs + 1), cudaMemcpyHostToDevice);
  Args a;
  a.one = cats[0];
  a.cats = static_cast<const Cat*>(P->d_cats);
  a.base = P->d_base;
  a.ncats = n_graphs;
  a.nb = nb;
  a.nconf = nconf;
  a.seg_cap = (o.variant & 1) ? 64 : kSegCap;
  a.force_hash = (o.variant & 1) ? 1 : 0;
  a.stage_cap = (o.variant & 2) ? 0 : kStageCap;
  a.hub_counter = P->counter;
  a.err = P->err;
  int max_deg = 0;
  for (int k = 0; k < n_graphs; ++k) max_deg = std::max(max_deg, graphs[k]->g.max_deg);
  const Count3Launch L = count3_launch(nb, nconf, kNone, !(o.variant & 4), false, false, max_deg);
  a.span_cap = (o.variant & 8) ? 2048 : L.span_cap;
  a.stage_alloc = L.stage_words;
  a.use_lut = (o.variant & 4) ? 0 : 1;
  a.compact = (o.variant & 32) ? 1 : 0;
  a.ring = 0;  // recorded plans keep the default walk
  a.first_wait_limit = (o.variant & 16) ? 0u : kWaitLimit;
  a.stage_cap = std::min(a.stage_cap, L.stage_words);
  void (*kern)(Args) = pick_count3<true>(kNone, true, L.smem_hist, L.lut);
  int per_sm = 0, sms = 0, dev = 0;
  if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, L.smem);
  cudaStream_t s = nullptr;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaMemsetAsync(P->counter, 0, sizeof(unsigned long long) + sizeof(int), s);
    for (int k = 0; k < n_graphs; ++k) cudaMemsetAsync(counts[k], 0, sizeof(uint64_t) * nconf, s);
    if (base[n_graphs] > 0) kern<<<std::max(1, per_sm) * sms, kThreads, L.smem, s>>>(a);
    cudaError_t ce = cudaStreamEndCapture(s, &P->graph);
    e = (e == cudaSuccess) ? ce : e;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&P->exec, P->graph, 0);
  if (s) cudaStreamDestroy(s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    gs_plan_destroy(P);
    return cuda_status(e);
  }
  *out = P;
  return GS_OK;
}

extern "C" int gs_plan_launch(gs_plan* P, void* stream) {
  if (!P || !P->exec) return GS_EINVAL;
  const cudaError_t e = cudaGraphLaunch(P->exec, static_cast<cudaStream_t>(stream));
  if (e == cudaSuccess) gs::note_launch();
  return gs::cuda_status(e);
}

extern "C" int gs_plan_wait(gs_plan* P, void* stream) {
  if (!P) return GS_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int herr = 0;
  cudaError_t e = cudaMemcpyAsync(&herr, P->err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return gs::cuda_status(e);
  return herr ? GS_ETIMEOUT : GS_OK;
}

extern "C" void gs_plan_destroy(gs_plan* P) {
  if (!P) return;
  if (P->exec) cudaGraphExecDestroy(P->exec);
  if (P->graph) cudaGraphDestroy(P->graph);
  cudaFree(P->d_cats);
  cudaFree(P->d_base);
  cudaFree(P->counter);
  delete P;
}

// ----------------------------------------------------------------------------
// Autotuning of the 3pCF launch choices. gs_tune_3pcf times the candidate
// variants on one hub shard of the caller's graph (a contiguous sample of
// about 1/16 of its edges) and remembers the fastest for graphs with the
// same bin count, weight mode and degree class; queries with variant -1
// use it (variant 0 when nothing has been tuned).
namespace gs {
namespace {
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, int> g_tuned;

std::tuple<int, int, int> tune_key(const Graph& g, int wmode) {
  const double mean = g.n ? (double)g.edges_total / (double)g.n : 0.0;
  int cls = 0;
  while (cls < 30 && (double)(1 << cls) < mean) ++cls;
  return {g.nb, wmode, cls};
}
}  // namespace

int resolve_variant(const Graph& g, int wmode, int variant) {
  if (variant >= 0) return variant;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tuned.find(tune_key(g, wmode));
  return it == g_tuned.end() ? 0 : it->second;
}
}  // namespace gs

extern "C" int gs_tune_3pcf(const gs_graph* G, const float* w, const gs_options* options,
                            int32_t* best_variant) {
  using namespace gs;
  if (!G || !best_variant) return GS_EINVAL;
  const Graph& g = G->g;
  Opts o = read_opts(options);
  const int nconf = (int)num_conf3(g.nb);
  const int wmode = w ? kExact : kNone;
  // the pair kernel (table or computed configuration ranks) and the
  // merge-walk kernel (512) with staged or global hub rows (2), table or
  // computed ranks (4), (weighted) per-warp hit compaction (32) and the
  // spoke-row prefetch ring (64)
  static const int kCandidates[10] = {0, 4, 512, 514, 516, 518, 544, 546, 576, 608};
  int best = 0;
  double best_ms = 1e300;
  int st = GS_OK;
  {
    Scratch sc(o.stream);
    FixedW fw;
    if (w) {
      st = prepare_weights(g, w, &fw, sc, o.stream);
      if (st) return st;
    }
    uint64_t* dc = sc.alloc<uint64_t>(nconf);
    double* dw = w ? sc.alloc<double>(nconf) : nullptr;
    if (!dc || (w && !dw)) return GS_ENOMEM;
    for (int c : kCandidates) {
      double ms = 0.0;
      for (int rep = 0; rep < 2 && !st; ++rep) {  // the first run warms caches up
        Opts t = o;
        t.variant = c;
        t.shard = 0;
        t.shards = 16;
        double k = 0.0;
        t.kernel_ms = &k;
        Scratch run(o.stream);
        st = count3_device(g, w ? &fw : nullptr, dc, dw, t, run);
        ms = k;
      }
      if (st) return st;
      if (ms < best_ms) {
        best_ms = ms;
        best = c;
      }
    }
  }
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tuned[tune_key(g, wmode)] = best;
  }
  *best_variant = best;
  return GS_OK;
}
