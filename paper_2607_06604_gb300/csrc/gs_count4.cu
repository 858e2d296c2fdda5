// Binned tetrahedron counts (Sec. 2.2) and the parity-decomposed channels
// (Sec. 3.2, Eq. volume), GB300 layout.
//
// A tetrahedron i < a < b < c is counted at its smallest vertex i. For hub i
// with m = |N+(i)| neighbours (local indices 0..m-1 in id order), a
// persistent CTA
//   1. stages N+(i) in shared memory with a bulk (TMA) copy, with the
//      minimum-image displacement of every neighbour from i;
//   2. builds the m x m bit matrix of adjacency within N+(i) (the paper's
//      per-hub connectivity matrix, Sec. 3.5.2, as bits) by testing every
//      pair (a, c), a < c, of staged displacements against the edge
//      distances, a ballot per 32-bit word;
//   3. for every triangle (a, b), b a bit of row a, takes the common bits
//      of rows a and b above b: each is a tetrahedron (i, a, b, c). This is
//      the three-way walk of Eq. (threeway) done 32 candidates per word.
// The six bins come from the staged row (hub edges) and from the staged
// displacements (the other three edges, recomputed exactly in integers).
// A table maps the raw bin tuple to its S4 orbit, the parity of one
// relabelling onto the orbit representative and the orbit's chirality; the
// signed volume is det[d_a, d_b, d_c] in 64-bit integers, multiplied by
// that parity. Counts use per-CTA shared-memory histograms flushed with
// 64-bit atomics. Hubs with more than kMaxSmemRow neighbours run in a
// second launch whose per-hub workspace lives in global scratch.
//
// When the per-orbit counters of every orbit do not fit in shared memory
// beside the hub workspace (unweighted: many bins; weighted: see below),
// shared memory holds the `hot` orbits only: the orbit tables are relabelled
// so that the orbits met most often in a sample of hubs come first, and a
// tetrahedron of any other orbit goes to the global counters directly.
//
// Weighted sums (exact, fixed-point W): the hub's sums of W_a W_b W_c are
// kept per orbit in shared 128-bit words (32-bit limbs), one for
// each sign of the volume so that a tetrahedron adds to one word only, and
// multiplied by W_i into the global 192-bit sums when the hub ends. Shared
// memory holds these words (and the counts) only for the `hot` orbits: the
// orbit tables are relabelled so that the orbits met most often in a
// sample of hubs come first, and a tetrahedron of any other orbit goes
// straight to the global sums with its full product.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>
#include <type_traits>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kThreads = 1024;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxSmemRow = 512;
// Squared-distance buckets for the bin lookup: bucket k covers
// [k 2^shift, (k + 1) 2^shift) with 2^shift no wider than the narrowest bin
// in squared distance, so a bucket holds at most one bin edge.
constexpr int kBucketMax = 2048;

struct Args {
  const int64_t* __restrict__ ptr;
  const int32_t* __restrict__ deg;
  const uint32_t* __restrict__ adj;  // row i at row_at(adj, ptr, i, adj_off, split, adj_off2)
  int64_t adj_off, split, adj_off2;
  int64_t hub_begin, hub_end;
  const int64_t* __restrict__ big;  // hubs above the shared capacity, taken first
  int64_t nbig;
  const int4* __restrict__ xyzp;
  const int64_t* __restrict__ e2g;
  const uint32_t* __restrict__ lut;
  int64_t n, box;
  int nb, n_orbits;
  int mcap;   // shared-memory workspace capacity (neighbours)
  int thr;    // hubs with more neighbours than this use the global workspace
  int gcap;   // global workspace capacity (neighbours)
  int bk_shift, bk_n;  // squared-distance buckets (bk_n = 0: binary search)
  int hot;             // orbits (slots) below this are accumulated in shared memory
  int64_t hub_stride;  // hubs hub_begin + k hub_stride (1: every hub)
  unsigned long long* even;
  unsigned long long* odd;
  unsigned long long* weven;  // [n_orbits][3] 192-bit
  unsigned long long* wodd;
  const int64_t* __restrict__ W;
  const uint8_t* __restrict__ pixsign;  // pixelised parity: 2-bit signs of sorted pixel triples
  unsigned long long* hub_counter;
  int* err;
  unsigned char* gscratch;  // per-CTA global workspace
  size_t gscratch_stride;
};

__device__ inline int64_t mi(int64_t d, int64_t box) {
  if (box) {
    if (2 * d >= box) d -= box;
    else if (2 * d < -box) d += box;
  }
  return d;
}

// Largest b with e2[b] <= D2 (the caller knows D2 is an edge): the bucket
// of D2 gives the bin of the bucket's start, and one comparison with the
// next edge finishes it; without buckets, a binary search.
template <class T>
__device__ inline int bin_of(T D2, const T* e2, int nb, const uint8_t* bk, int shift) {
  if (bk) {
    const int b = bk[(uint64_t)D2 >> shift];
    return b + (D2 >= e2[b + 1] ? 1 : 0);
  }
  int lo = 0, hi = nb;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (e2[mid] <= D2) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Squared distance between two hub-relative displacements. With
// SMALLR (E_nb < 2^15) every component of an edge is below 2^15 and the sum
// below 2^32, so 32-bit arithmetic is exact.
template <bool SMALLR>
__device__ inline auto d2(const int4& p, const int4& q) {
  if constexpr (SMALLR) {
    const int x = q.x - p.x, y = q.y - p.y, z = q.z - p.z;
    return (uint32_t)(x * x) + (uint32_t)(y * y) + (uint32_t)(z * z);
  } else {
    const int64_t x = (int64_t)q.x - p.x, y = (int64_t)q.y - p.y, z = (int64_t)q.z - p.z;
    return x * x + y * y + z * z;
  }
}

// det[da, db, dc] exactly. With SMALLR the 2x2 minors fit in 32 bits.
template <bool SMALLR>
__device__ inline int64_t det3(const int4& da, const int4& db, const int4& dc) {
  if constexpr (SMALLR) {
    const int m0 = db.y * dc.z - db.z * dc.y;
    const int m1 = db.x * dc.z - db.z * dc.x;
    const int m2 = db.x * dc.y - db.y * dc.x;
    return (int64_t)da.x * m0 - (int64_t)da.y * m1 + (int64_t)da.z * m2;
  } else {
    return (int64_t)da.x * ((int64_t)db.y * dc.z - (int64_t)db.z * dc.y) -
           (int64_t)da.y * ((int64_t)db.x * dc.z - (int64_t)db.z * dc.x) +
           (int64_t)da.z * ((int64_t)db.x * dc.y - (int64_t)db.y * dc.x);
  }
}

// Direction pixel of the pixelised parity channel (Sec. 3.2 stores one
// pixel byte per spoke and treats |V| < 1e-9 as degenerate; the scheme is
// fixed here as 256 equal-area pixels): 16 bands of width 1/8 in
// cos(theta) = z / |d| (a direction on a band edge belongs to the band
// above it) times 16 sectors of pi / 8 in phi = atan2(y, x) in [0, 2 pi)
// (an edge belongs to the sector above it; sector 0 on the z axis); pixel =
// 16 band + sector. Everything is decided with exact 64-bit integer
// comparisons: z / |d| against s / 8 through 64 z^2 against s^2 |d|^2, and
// phi within its quadrant against pi/8, pi/4, 3pi/8 through tan(pi/8) =
// sqrt(2) - 1 and tan(3pi/8) = sqrt(2) + 1 squared out.
__host__ __device__ inline int dir_pixel(int64_t x, int64_t y, int64_t z) {
  // band = 8 + floor(8 z / |d|), at most 15. On the device t = 8 z / |d| is
  // first formed in single precision (relative error below 8 2^-24 from the
  // conversions, products, sums and the reciprocal square root's 2 ulp, so
  // below 2^-18 absolutely): at least 2^-10 from every integer, its floor is
  // exact; otherwise (and for d = 0) the integer comparisons decide.
  int band = -1;
#ifdef __CUDA_ARCH__
  {
    // the components fit 32 bits (displacements below 2^20): 32-bit
    // conversions, not the FP64 pipe's 64-bit ones
    const float fx = (float)(int)x, fy = (float)(int)y, fz = (float)(int)z;
    const float t = 8.0f * fz * rsqrtf(fx * fx + fy * fy + fz * fz);
    if (fabsf(t - rintf(t)) >= 0.0009765625f) {
      const int f = 8 + (int)floorf(t);
      band = f < 0 ? 0 : (f > 15 ? 15 : f);
    }
  }
#endif
  if (band < 0) {
    const int64_t n2 = x * x + y * y + z * z, z64 = 64 * z * z;
    band = z >= 0 ? 8 : 0;
    for (int s = 1; s <= 7; ++s) {
      const int64_t edge = (int64_t)(s * s) * n2;
      // z >= 0: edges s/8 at or below z/|d|; z < 0: edges -s/8 at or below it
      band += (z >= 0 ? (z64 >= edge) : (z64 <= edge)) ? 1 : 0;
    }
  }
  int sector = 0;
  if (x != 0 || y != 0) {
    // turn by -pi/2 until the direction lies in [0, pi/2): a > 0, b >= 0
    int quarter;
    int64_t a, b;
    if (x > 0 && y >= 0) {
      quarter = 0, a = x, b = y;
    } else if (x <= 0 && y > 0) {
      quarter = 1, a = y, b = -x;
    } else if (x < 0 && y <= 0) {
      quarter = 2, a = -x, b = -y;
    } else {
      quarter = 3, a = -y, b = x;
    }
    // phi >= pi/8 iff b >= (sqrt 2 - 1) a, phi >= 3 pi/8 iff b >= (sqrt 2 + 1) a
    // (never equal for integers, a > 0); on the device b - k a is formed in
    // single precision (a, b below 2^21: error below 1/2) and decides when
    // at least 1 from zero; otherwise, and on the host, the squared integer
    // forms decide
    int e1 = -1, e3 = -1;
#ifdef __CUDA_ARCH__
    if (a < (int64_t(1) << 21) && b < (int64_t(1) << 21)) {
      const float fa = (float)(int)a, fb = (float)(int)b;
      const float g1 = fmaf(-0.41421356237f, fa, fb), g3 = fmaf(-2.41421356237f, fa, fb);
      if (fabsf(g1) >= 1.0f) e1 = g1 > 0.0f ? 1 : 0;
      if (fabsf(g3) >= 1.0f) e3 = g3 > 0.0f ? 1 : 0;
    }
#endif
    const int64_t a2 = 2 * a * a;
    if (e1 < 0) e1 = ((a + b) * (a + b) >= a2) ? 1 : 0;
    if (e3 < 0) e3 = (b > a && (b - a) * (b - a) >= a2) ? 1 : 0;
    sector = 4 * quarter + e1 + (b >= a ? 1 : 0) + e3;
  }
  return 16 * band + sector;
}

// Sign of the pixel volume (u_p1 x u_p2) . u_p3 of three pixel centres: 0
// for repeated pixels, else the table entry of the sorted triple times the
// parity of the sort. The table (host-built in FP64, 0 where |V| < 1e-9)
// holds two bits per sorted triple p < q < r (1: positive, 2: negative, 0:
// degenerate), entry C(r,3) + C(q,2) + p, four to a byte (690 KB).
__device__ inline int pix_sign(const uint8_t* __restrict__ T, int p1, int p2, int p3) {
  if (p1 == p2 || p1 == p3 || p2 == p3) return 0;
  int s = 1;
  if (p1 > p2) { const int t = p1; p1 = p2; p2 = t; s = -s; }
  if (p2 > p3) { const int t = p2; p2 = p3; p3 = t; s = -s; }
  if (p1 > p2) { const int t = p1; p1 = p2; p2 = t; s = -s; }
  const int idx = p3 * (p3 - 1) * (p3 - 2) / 6 + p2 * (p2 - 1) / 2 + p1;
  const int code = (T[idx >> 2] >> ((idx & 3) << 1)) & 3;
  return s * ((code & 1) - (code >> 1));
}

// A 128-bit two's complement value (lo, hi) into a shared 128-bit sum kept
// as four 32-bit limbs, least significant first (sums modulo 2^128; the
// caller keeps the true sum in range). 32-bit shared atomics are native;
// the carries ripple through the returned old values, and a limb whose
// addend (with the carry in) is zero is skipped. (64-bit shared atomic adds
// measured 2.3 times slower in the triangle kernel's record.)
__device__ inline void shared_add_i128(unsigned long long* p64, unsigned long long lo,
                                       unsigned long long hi) {
  unsigned* p = reinterpret_cast<unsigned*>(p64);
  const uint32_t x0 = (uint32_t)lo, x1 = (uint32_t)(lo >> 32), x2 = (uint32_t)hi,
                 x3 = (uint32_t)(hi >> 32);
  uint32_t o = atomicAdd(p, x0);
  uint32_t c = (o + x0 < o) ? 1u : 0u;
  const uint32_t s1 = x1 + c;
  c = (s1 < x1) ? 1u : 0u;  // x1 = 2^32 - 1 and a carry: s1 = 0
  if (s1) {
    o = atomicAdd(p + 1, s1);
    c |= (o + s1 < o) ? 1u : 0u;
  }
  const uint32_t s2 = x2 + c;
  c = (s2 < x2) ? 1u : 0u;
  if (s2) {
    o = atomicAdd(p + 2, s2);
    c |= (o + s2 < o) ? 1u : 0u;
  }
  const uint32_t s3 = x3 + c;
  if (s3) atomicAdd(p + 3, s3);
}

// A 192-bit two's complement value into three global 64-bit words.
__device__ inline void atomic_add_w192(unsigned long long* g, unsigned long long w0,
                                       unsigned long long w1, unsigned long long w2) {
  const unsigned long long o0 = atomicAdd(g, w0);
  const unsigned long long c0 = (o0 + w0 < o0) ? 1ull : 0ull;
  const unsigned long long s1 = w1 + c0;
  const unsigned long long c1a = (s1 < w1) ? 1ull : 0ull;  // w1 = 2^64 - 1 and a carry
  unsigned long long c1b = 0;
  if (s1) {
    const unsigned long long o1 = atomicAdd(g + 1, s1);
    c1b = (o1 + s1 < o1) ? 1ull : 0ull;
  }
  const unsigned long long s2 = w2 + c1a + c1b;
  if (s2) atomicAdd(g + 2, s2);
}

// S * Wi into a global 192-bit sum: S a signed 128-bit hub sum (lo, hi),
// |Wi| < 2^63.
__device__ inline void fold_i128(unsigned long long* g, unsigned long long lo,
                                 unsigned long long hi, long long Wi) {
  const bool sn = (long long)hi < 0, wn = Wi < 0;
  if (sn) {
    lo = ~lo + 1ull;
    hi = ~hi + (lo == 0ull ? 1ull : 0ull);
  }
  const unsigned long long v = wn ? (unsigned long long)(-Wi) : (unsigned long long)Wi;
  unsigned long long p0 = lo * v;
  const unsigned long long t = __umul64hi(lo, v);
  unsigned long long p1 = hi * v + t;
  unsigned long long p2 = __umul64hi(hi, v) + (p1 < t ? 1ull : 0ull);
  if (sn != wn) {
    p0 = ~p0 + 1ull;
    unsigned long long c = p0 == 0ull ? 1ull : 0ull;
    p1 = ~p1 + c;
    c = (c && p1 == 0ull) ? 1ull : 0ull;
    p2 = ~p2 + c;
  }
  atomic_add_w192(g, p0, p1, p2);
}

struct Workspace {
  uint32_t* row;      // staged N+(i) words
  int4* disp;         // displacement of each neighbour from the hub
  uint32_t* bits;     // m x W bit matrix
  int* cid;           // caller index of each neighbour (pixelised parity)
  int* wv;            // weight of each neighbour (weighted sums)
  uint8_t* brow;      // per warp: bin(a, c) of its current row a, cap bytes each
  uint8_t* prow;      // pixelised parity, per warp: pixel of D_c - D_a for row a
  uint32_t* queue;    // per-warp queue of (b, c) entries: kWarps x 64 words
  int cap;
};

__device__ inline Workspace carve(unsigned char* p, int cap, bool pix) {
  const int Wc = (cap + 31) / 32;
  Workspace w;
  w.row = reinterpret_cast<uint32_t*>(p);
  p += (size_t)pad_row(cap) * 4;
  w.disp = reinterpret_cast<int4*>(p);
  p += (size_t)cap * 16;
  w.bits = reinterpret_cast<uint32_t*>(p);
  p += (size_t)cap * Wc * 4;
  w.cid = reinterpret_cast<int*>(p);
  p += (size_t)cap * 4;
  w.wv = reinterpret_cast<int*>(p);
  p += (size_t)cap * 4;
  w.brow = reinterpret_cast<uint8_t*>(p);
  p += (size_t)kWarps * ((cap + 15) & ~15);
  w.prow = reinterpret_cast<uint8_t*>(p);
  if (pix) p += (size_t)kWarps * ((cap + 15) & ~15);
  w.queue = reinterpret_cast<uint32_t*>(p);
  w.cap = (cap + 15) & ~15;
  return w;
}

// One hub: stage N+(i), build the neighbour bit matrix, enumerate the
// tetrahedra. GW: the workspace is in global memory (rows above the shared
// capacity) and counts go straight to the global histograms. Returns false
// when the staging copy timed out.
// Shared cells per weighted slot: one (no parity) or three (V = 0, V > 0,
// V < 0), each a u32 count and a 128-bit sum; even = all three, odd = the
// second minus the third.
template <bool PARITY>
constexpr int kCat = PARITY ? 3 : 1;

// h_even / h_odd: unweighted per-orbit counts; weighted, h_even holds the
// cells' counts and h_sum their sums.
template <bool PARITY, bool WEIGHTED, bool SMALLR, bool GW, bool PIX, class E2T>
__device__ bool hub4(const Args& a, const Workspace& w, const E2T* e2, const uint8_t* bk,
                     unsigned* h_even, int* h_odd, unsigned long long* h_sum, int64_t i, int m,
                     uint64_t* bar, uint32_t& phase, int* s_row) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nb = a.nb;
  const int W = (m + 31) / 32;
  const uint32_t* grow = row_at(a.adj, a.ptr, i, a.adj_off, a.split, a.adj_off2);
  const uint32_t* row = w.row;
  if (!GW) {
    if (tid == 0) bulk_load(w.row, grow, (uint32_t)pad_row(m) * 4u, bar);
  } else {
    row = grow;
  }
  for (int k = tid; k < m * W; k += kThreads) w.bits[k] = 0u;
  if (!GW) {
    const bool ok = mbar_wait(bar, phase, kWaitLimit);
    if (__syncthreads_or(!ok)) {
      // report, then wait (bounded) for the copy to land before giving up
      if (tid == 0) atomicOr(a.err, kErrTimeout);
      if (!ok) mbar_wait(bar, phase, kWaitLimit);
      __syncthreads();
      return false;
    }
    phase ^= 1u;
  } else {
    __syncthreads();
  }
  const int4 P = a.xyzp[i];
  for (int k = tid; k < m; k += kThreads) {
    const uint32_t id = edge_id(row[k]);
    const int4 Q = a.xyzp[id];
    // the fourth component carries the hub edge's bin, so one 128-bit load
    // gives a vertex's displacement and b_i,vertex
    const int dx = (int)mi((int64_t)Q.x - P.x, a.box), dy = (int)mi((int64_t)Q.y - P.y, a.box),
              dz = (int)mi((int64_t)Q.z - P.z, a.box);
    w.disp[k] = make_int4(dx, dy, dz, (int)edge_bin(row[k]));
    // pixelised parity: the caller index (below 2^24) and, in the top byte,
    // the pixel of the spoke from the hub
    if (PIX) w.cid[k] = (int)((unsigned)Q.w | ((unsigned)dir_pixel(dx, dy, dz) << 24));
    if (WEIGHTED) w.wv[k] = (int)a.W[id];
  }
  __syncthreads();
  if (tid == 0) *s_row = 0;
  // bit matrix: row a gets bit c for every c > a whose distance from a is an
  // edge's, E_0^2 <= |D_c - D_a|^2 < E_nb^2 on the staged hub-relative
  // displacements (4 E_nb < L makes their difference the pair's minimum
  // image); a warp per row, a ballot per 32-bit word
  const int64_t e2lo = (int64_t)e2[0], e2hi = (int64_t)e2[nb];
  for (int sa = warp; sa < m - 1; sa += kWarps) {
    const int4 da = w.disp[sa];
    for (int c0 = (sa + 1) & ~31; c0 < m; c0 += 32) {
      const int c = c0 + lane;
      bool edge = false;
      if (c > sa && c < m) {
        const int4 dc = w.disp[c];
        const int x = dc.x - da.x, y = dc.y - da.y, z = dc.z - da.z;
        const long long D2 = (long long)x * x + (long long)y * y + (long long)z * z;
        edge = D2 >= e2lo && D2 < e2hi;
      }
      const uint32_t word = __ballot_sync(0xffffffffu, edge);
      if (lane == 0) w.bits[sa * W + (c0 >> 5)] = word;
    }
  }
  __syncthreads();
  // tetrahedra: warp per row a, triangles (a, b) in a warp-uniform loop;
  // the common neighbours c > b of a and b are compacted into a per-warp
  // queue of (b, c) entries that carries over between triangles, and each
  // batch of 32 entries is processed one tetrahedron per lane
  const int64_t Wi = WEIGHTED ? a.W[i] : 0;
  uint32_t* qbc = w.queue + warp * 64;
  // rows near the start of N+(i) carry most of the work: warps take rows
  // from a shared counter (reset by thread 0 before the bit matrix was built)
  for (;;) {
    int sa = 0;
    if (lane == 0) sa = atomicAdd(s_row, 1);
    sa = __shfl_sync(0xffffffffu, sa, 0);
    if (sa >= m - 2) break;
    const uint32_t wa = row[sa];
    const int b01 = (int)edge_bin(wa);
    const int4 da = w.disp[sa];
    const int64_t Wa = WEIGHTED ? (int64_t)w.wv[sa] : 0;
    const int64_t Wia = Wi * Wa;
    const uint32_t* bra = w.bits + sa * W;
    // bin(a, c) of every edge (a, c) of the row, once per row: the triangle
    // loop and the drain read b_12 and b_13 from here
    uint8_t* brw = w.brow + (size_t)warp * w.cap;
    // pixelised parity: the pixels of the spokes from a (to the hub and to
    // every c of the row), used when a has the smallest caller index
    uint8_t* prw = w.prow + (size_t)warp * w.cap;
    int pneg = 0;
    for (int c = sa + 1 + lane; c < m; c += 32)
      if ((bra[c >> 5] >> (c & 31)) & 1u) {
        const int4 dc = w.disp[c];
        brw[c] = (uint8_t)bin_of(d2<SMALLR>(da, dc), e2, nb, bk, a.bk_shift);
        if (PIX)
          prw[c] = (uint8_t)dir_pixel((int64_t)dc.x - da.x, (int64_t)dc.y - da.y,
                                      (int64_t)dc.z - da.z);
      }
    if (PIX) pneg = dir_pixel(-(int64_t)da.x, -(int64_t)da.y, -(int64_t)da.z);
    __syncwarp();
    // the warp's queue of (b, c) entries is a ring of 64 slots: entries
    // [qh, qt) are pending; a drain takes the 32 (or, at the end of the row,
    // all) oldest, one per lane
    int qh = 0, qt = 0;
    auto drain = [&](bool all) {
      if (qt - qh >= 32 || (all && qt > qh)) {
        const int take = qt - qh < 32 ? qt - qh : 32;  // warp-uniform
        const bool active = lane < take;
        __syncwarp();  // the entries written by other lanes are visible
        const uint32_t e = active ? qbc[(qh + lane) & 63] : 0u;
        __syncwarp();  // read before any lane writes the next entries
        qh += take;
        if (active) {
          const int sb = (int)(e >> 16), sc = (int)(e & 0xFFFFu);
          const int b12 = brw[sb];
          const int4 db = w.disp[sb], dc = w.disp[sc];
          const int b02 = db.w, b03 = dc.w;
          const int b13 = brw[sc];
          const int b23 = bin_of(d2<SMALLR>(db, dc), e2, nb, bk, a.bk_shift);
          const uint32_t ent =
              a.lut[(((uint32_t)((b01 * nb + b02) * nb + b12) * nb + b03) * nb + b13) * nb + b23];
          const int orbit = (int)(ent & 0x3FFFFFFFu);
          // the volume's sign, relabelled onto the orbit representative (0:
          // achiral orbit or degenerate tetrahedron)
          int sgn = 0;
          if (PARITY && (ent >> 31)) {
            if constexpr (PIX) {
              // the pixelised reading: the three spokes from the vertex with
              // the smallest caller index, taken in ascending caller order; a
              // sorting network orders the vertices (0 = hub, 1 = a, 2 = b,
              // 3 = c) and keeps the parity of the reordering
              const int ca = w.cid[sa], cb = w.cid[sb], cc = w.cid[sc];
              int key[4] = {P.w, ca & 0xFFFFFF, cb & 0xFFFFFF, cc & 0xFFFFFF};
              int vx[4] = {0, 1, 2, 3};
              int par = 1;
              auto cx = [&](int u, int v) {
                if (key[u] > key[v]) {
                  const int tk = key[u];
                  key[u] = key[v];
                  key[v] = tk;
                  const int tv = vx[u];
                  vx[u] = vx[v];
                  vx[v] = tv;
                  par = -par;
                }
              };
              cx(0, 1);
              cx(2, 3);
              cx(0, 2);
              cx(1, 3);
              cx(1, 2);
              // pixel of the spoke from the origin o to each vertex, and
              // whether a spoke has zero length (coincident points)
              const int o = vx[0];
              int p0 = 0, p1 = 0, p2 = 0, p3 = 0;
              bool zero;
              auto same = [](const int4& u, const int4& v) {
                return u.x == v.x && u.y == v.y && u.z == v.z;
              };
              if (o == 0) {  // from the hub: cached with the caller indices
                p1 = (int)((unsigned)ca >> 24);
                p2 = (int)((unsigned)cb >> 24);
                p3 = (int)((unsigned)cc >> 24);
                zero = (da.x == 0 && da.y == 0 && da.z == 0) ||
                       (db.x == 0 && db.y == 0 && db.z == 0) ||
                       (dc.x == 0 && dc.y == 0 && dc.z == 0);
              } else if (o == 1) {  // from a: the row's cached pixels
                p0 = pneg;
                p2 = prw[sb];
                p3 = prw[sc];
                zero = (da.x == 0 && da.y == 0 && da.z == 0) || same(db, da) || same(dc, da);
              } else {  // from b or c: three pixelisations
                const int4 Do = o == 2 ? db : dc, Dq = o == 2 ? dc : db;
                const int q0 = dir_pixel(-(int64_t)Do.x, -(int64_t)Do.y, -(int64_t)Do.z);
                const int q1 = dir_pixel((int64_t)da.x - Do.x, (int64_t)da.y - Do.y,
                                         (int64_t)da.z - Do.z);
                const int qq = dir_pixel((int64_t)Dq.x - Do.x, (int64_t)Dq.y - Do.y,
                                         (int64_t)Dq.z - Do.z);
                p0 = q0;
                p1 = q1;
                if (o == 2) p3 = qq;
                else p2 = qq;
                zero = (Do.x == 0 && Do.y == 0 && Do.z == 0) || same(da, Do) || same(Dq, Do);
              }
              auto pix_of = [&](int v) { return v == 0 ? p0 : (v == 1 ? p1 : (v == 2 ? p2 : p3)); };
              const int px[3] = {pix_of(vx[1]), pix_of(vx[2]), pix_of(vx[3])};
              sgn = zero ? 0 : par * pix_sign(a.pixsign, px[0], px[1], px[2]);
            } else {
              const int64_t V = det3<SMALLR>(da, db, dc);
              sgn = V > 0 ? 1 : (V < 0 ? -1 : 0);
            }
            if ((ent >> 30) & 1u) sgn = -sgn;
          }
          // orbits below a.hot live in shared memory (every orbit when
          // unweighted)
          const bool hot = !GW && orbit < a.hot;
          if (WEIGHTED) {
            const int64_t Wbc = (int64_t)w.wv[sb] * w.wv[sc];  // below 2^60
            long long plo, phi;
            if (hot) {
              // the hub's count and sum of W_a W_b W_c (below 2^90) in the
              // orbit's cell for V = 0 / V > 0 / V < 0
              const int cell = kCat<PARITY> * orbit + (sgn > 0 ? 1 : (sgn < 0 ? 2 : 0));
              atomicAdd(h_even + cell, 1u);
              mul_i128(Wa, Wbc, &plo, &phi);
              shared_add_i128(h_sum + 2 * cell, (unsigned long long)plo, (unsigned long long)phi);
            } else {
              // (W_i W_a)(W_b W_c) straight into the global sums
              atomicAdd(a.even + orbit, 1ull);
              mul_i128(Wia, Wbc, &plo, &phi);
              unsigned long long lo = (unsigned long long)plo, hi = (unsigned long long)phi;
              atomic_add_i192(a.weven + 3 * orbit, lo, hi);
              if (PARITY && sgn != 0) {
                atomicAdd(a.odd + orbit, (unsigned long long)(long long)sgn);
                if (sgn < 0) {  // negate the 128-bit product
                  lo = ~lo + 1ull;
                  hi = ~hi + (lo == 0ull ? 1ull : 0ull);
                }
                atomic_add_i192(a.wodd + 3 * orbit, lo, hi);
              }
            }
          } else {
            if (hot) atomicAdd(h_even + orbit, 1u);
            else atomicAdd(a.even + orbit, 1ull);
            if (PARITY && sgn != 0) {
              if (hot) atomicAdd(h_odd + orbit, sgn);
              else atomicAdd(a.odd + orbit, (unsigned long long)(long long)sgn);
            }
          }
        }
      }
    };
    for (int wb0 = sa >> 5; wb0 < W; ++wb0) {
      uint32_t xb = bra[wb0];
      while (xb) {  // warp-uniform: every lane walks the same bits
        const int sb = wb0 * 32 + __ffs(xb) - 1;
        xb &= xb - 1u;
        const uint32_t* brb = w.bits + sb * W;
        for (int wc = sb >> 5; wc < W; ++wc) {
          uint32_t x = bra[wc] & brb[wc];
          if (wc == (sb >> 5)) x &= ~((2u << (sb & 31)) - 1u);
          if (!x) continue;
          const bool set = (x >> lane) & 1u;
          if (set)
            qbc[(qt + __popc(x & ((1u << lane) - 1u))) & 63] =
                ((uint32_t)sb << 16) | (uint32_t)(wc * 32 + lane);
          qt += __popc(x);  // at most 31 + 32 pending: the ring never overfills
          drain(false);
        }
      }
    }
    drain(true);
  }
  __syncthreads();
  return true;
}

template <bool PARITY, bool WEIGHTED, bool SMALLR, bool PIX>
__global__ void __launch_bounds__(kThreads, 1) k_count4(Args a) {
  extern __shared__ __align__(16) unsigned char smem[];
  using E2T = typename std::conditional<SMALLR, uint32_t, int64_t>::type;
  __shared__ uint64_t bar;
  __shared__ int64_t s_hub;
  __shared__ int s_flush;
  __shared__ unsigned long long s_pending;
  __shared__ E2T e2[kMaxBins4 + 1];
  __shared__ uint8_t s_bk[kBucketMax];
  __shared__ int s_row;

  const int tid = threadIdx.x;
  // shared slots of the orbits below a.hot: unweighted, the even and odd
  // counts; weighted, kCat cells of a 128-bit sum (the hub's) and a count
  const int nh = a.hot;
  constexpr int nc = WEIGHTED ? kCat<PARITY> : 1;
  unsigned char* sp = smem;
  unsigned long long* h_sum = reinterpret_cast<unsigned long long*>(sp);
  sp += WEIGHTED ? (size_t)nh * nc * 16 : 0;
  unsigned* h_even = reinterpret_cast<unsigned*>(sp);
  sp += (size_t)nh * nc * 4;
  int* h_odd = reinterpret_cast<int*>(sp);
  sp += (PARITY && !WEIGHTED) ? (size_t)nh * 4 : 0;
  unsigned char* sws = reinterpret_cast<unsigned char*>(((uintptr_t)sp + 15) & ~(uintptr_t)15);
  const Workspace ws_s = carve(sws, a.mcap, PIX);
  const Workspace ws_g = carve(a.gscratch ? a.gscratch + (size_t)blockIdx.x * a.gscratch_stride
                                          : sws,
                               a.gscratch ? a.gcap : a.mcap, PIX);

  for (int k = tid; k < nh * nc; k += kThreads) {
    h_even[k] = 0;
    if (PARITY && !WEIGHTED) h_odd[k] = 0;
    if (WEIGHTED) h_sum[2 * k] = h_sum[2 * k + 1] = 0ull;
  }
  for (int b = tid; b <= a.nb; b += kThreads) e2[b] = (E2T)a.e2g[b];
  for (int k = tid; k < a.bk_n; k += kThreads) {
    const int64_t x = (int64_t)k << a.bk_shift;
    int b = 0;
    while (b + 1 < a.nb && a.e2g[b + 1] <= x) ++b;
    s_bk[k] = (uint8_t)b;
  }
  const uint8_t* bk = a.bk_n ? s_bk : nullptr;
  if (tid == 0) {
    mbar_init(&bar, 1);
    s_pending = 0;
  }
  __syncthreads();
  uint32_t phase = 0;

  auto flush = [&]() {
    for (int k = tid; k < nh; k += kThreads) {
      if (WEIGHTED) {
        // cells V = 0, V > 0, V < 0: even = all three, odd = second - third
        const unsigned c0 = h_even[nc * k];
        const unsigned cp = PARITY ? h_even[nc * k + 1] : 0u;
        const unsigned cn = PARITY ? h_even[nc * k + 2] : 0u;
        if (c0 | cp | cn) {
          atomicAdd(a.even + k, (unsigned long long)c0 + cp + cn);
          if (PARITY && cp != cn)
            atomicAdd(a.odd + k, (unsigned long long)((long long)cp - (long long)cn));
          h_even[nc * k] = 0;
          if (PARITY) h_even[nc * k + 1] = h_even[nc * k + 2] = 0;
        }
        continue;
      }
      const unsigned c = h_even[k];
      if (c) {
        atomicAdd(a.even + k, (unsigned long long)c);
        h_even[k] = 0;
      }
      if (PARITY) {
        const int o = h_odd[k];
        if (o) {
          atomicAdd(a.odd + k, (unsigned long long)(long long)o);
          h_odd[k] = 0;
        }
      }
    }
  };

  for (;;) {
    if (tid == 0) {
      // the long rows first (they are few and slow), then every other hub
      const int64_t q = (int64_t)atomicAdd(a.hub_counter, 1ull);
      int64_t i;
      int d = 0;
      if (q < a.nbig) {
        i = a.big[q];
        d = a.deg[i];
      } else {
        int64_t qq = q - a.nbig;
        for (;;) {
          i = a.hub_begin + qq * a.hub_stride;
          d = (i < a.hub_end) ? a.deg[i] : 0;
          if (i >= a.hub_end || (d >= 3 && d <= a.thr)) break;
          qq = (int64_t)atomicAdd(a.hub_counter, 1ull) - a.nbig;
        }
      }
      s_hub = i;
      s_flush = 0;
      if (i < a.hub_end && d <= a.thr) {
        const unsigned long long m = (unsigned long long)d;
        const unsigned long long need = m * (m - 1) * (m - 2) / 6;
        if (s_pending + need > 0x7FFFFFFFull) {
          s_flush = 1;
          s_pending = need;
        } else {
          s_pending += need;
        }
      }
    }
    __syncthreads();
    const int64_t i = s_hub;
    if (i >= a.hub_end) break;
    if (s_flush) {
      flush();
      __syncthreads();
    }
    const int m = a.deg[i];
    bool ok;
    if (m > a.thr) {
      ok = hub4<PARITY, WEIGHTED, SMALLR, true, PIX>(a, ws_g, e2, bk, h_even, h_odd, h_sum, i, m,
                                                     &bar, phase, &s_row);
    } else {
      ok = hub4<PARITY, WEIGHTED, SMALLR, false, PIX>(a, ws_s, e2, bk, h_even, h_odd, h_sum, i,
                                                      m, &bar, phase, &s_row);
      if (WEIGHTED && ok) {
        // the hub's sums times W_i into the global 192-bit sums (the
        // barrier at the top of the loop orders the clearing before the
        // next hub's additions)
        const long long Wi = a.W[i];
        for (int k = tid; k < nh; k += kThreads) {
          unsigned long long* c = h_sum + 2 * nc * k;
          unsigned long long elo = c[0], ehi = c[1], olo = 0, ohi = 0;
          if (PARITY) {
            // even = S0 + S+ + S-, odd = S+ - S- (each below 2^115 in
            // magnitude, so no 128-bit overflow)
            const unsigned long long plo = c[2], phi = c[3], nlo = c[4], nhi = c[5];
            unsigned long long t = elo + plo;
            ehi += phi + (t < elo ? 1ull : 0ull);
            elo = t;
            t = elo + nlo;
            ehi += nhi + (t < elo ? 1ull : 0ull);
            elo = t;
            olo = plo - nlo;
            ohi = phi - nhi - (plo < nlo ? 1ull : 0ull);
            c[2] = c[3] = c[4] = c[5] = 0ull;
          }
          c[0] = c[1] = 0ull;
          if (elo | ehi) fold_i128(a.weven + 3 * k, elo, ehi, Wi);
          if (PARITY && (olo | ohi)) fold_i128(a.wodd + 3 * k, olo, ohi, Wi);
        }
      }
    }
    if (!ok) return;
  }
  __syncthreads();
  flush();
}

size_t workspace_bytes(int mcap, bool pix) {
  const size_t Wc = (size_t)(mcap + 31) / 32;
  return (size_t)pad_row(mcap) * 4 + (size_t)mcap * 16 + (size_t)mcap * Wc * 4 +
         (size_t)mcap * 8 + (size_t)kWarps * ((mcap + 15) & ~15) * (pix ? 2 : 1) +
         (size_t)kWarps * 64 * 5 + 64;
}

}  // namespace

__global__ void k_i192_to_double(const unsigned long long* acc, int64_t n, int scale, double* out);
__global__ void k_u64_to_double(const unsigned long long* c, int64_t n, double* out);
__global__ void k_i64_to_double(const long long* c, int64_t n, double* out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    out[k] = (double)c[k];
}

namespace {
// Signs of the pixel volume of every sorted pixel triple p < q < r (0 below
// 1e-9 in magnitude), built once on the host in FP64 and copied to each
// device on first use.
std::mutex g_pix_mu;
std::vector<uint8_t> g_pix_host;  // 2 bits per sorted triple
uint8_t* g_pix_dev[64] = {nullptr};

const uint8_t* pixel_sign_table(int* status) {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) {
    *status = GS_ERANGE;
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(g_pix_mu);
  if (g_pix_dev[dev]) return g_pix_dev[dev];
  if (g_pix_host.empty()) {
    double u[256][3];
    for (int p = 0; p < 256; ++p) {
      const double zc = (2.0 * (p >> 4) + 1.0) / 16.0 - 1.0;
      const double phi = M_PI * (2.0 * (p & 15) + 1.0) / 16.0;
      const double rho = std::sqrt((1.0 - zc) * (1.0 + zc));
      u[p][0] = rho * std::cos(phi);
      u[p][1] = rho * std::sin(phi);
      u[p][2] = zc;
    }
    g_pix_host.assign(((size_t)256 * 255 * 254 / 6 + 3) / 4, 0);
    size_t idx = 0;
    for (int r = 0; r < 256; ++r)
      for (int q = 0; q < r; ++q)
        for (int p = 0; p < q; ++p, ++idx) {
          const double* a = u[p];
          const double* b = u[q];
          const double* c = u[r];
          const double v = (a[1] * b[2] - a[2] * b[1]) * c[0] + (a[2] * b[0] - a[0] * b[2]) * c[1] +
                           (a[0] * b[1] - a[1] * b[0]) * c[2];
          const unsigned code = std::fabs(v) < 1e-9 ? 0u : (v > 0 ? 1u : 2u);
          g_pix_host[idx >> 2] |= (uint8_t)(code << ((idx & 3) << 1));
        }
  }
  uint8_t* d = nullptr;
  cudaError_t e = cudaMalloc(&d, g_pix_host.size());
  if (e == cudaSuccess) e = cudaMemcpy(d, g_pix_host.data(), g_pix_host.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (d) cudaFree(d);
    *status = cuda_status(e);
    return nullptr;
  }
  g_pix_dev[dev] = d;
  return d;
}

// Orbit table relabelled to slots: orbit o becomes slot_of[o], flags kept.
__global__ void k_relabel_lut(const uint32_t* __restrict__ lut, int64_t n,
                              const int32_t* __restrict__ slot_of, uint32_t* out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t e = lut[k];
    out[k] = (e & 0xC0000000u) | (uint32_t)slot_of[e & 0x3FFFFFFFu];
  }
}

// Per-slot results back to orbit order: dst[o] = src[slot_of[o]], `words`
// 64-bit words per entry.
__global__ void k_slots_to_orbits(const unsigned long long* __restrict__ src,
                                  const int32_t* __restrict__ slot_of, int64_t n, int words,
                                  unsigned long long* dst) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n * words;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = k / words;
    dst[k] = src[(int64_t)slot_of[o] * words + (k - o * words)];
  }
}

__global__ void k_dir_pixels(const int32_t* d, int64_t n, uint8_t* out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    out[k] = (uint8_t)dir_pixel(d[3 * k], d[3 * k + 1], d[3 * k + 2]);
}
}  // namespace

int direction_pixels_device(const int32_t* d_dirs, int64_t n, uint8_t* d_out, cudaStream_t s) {
  if (n > 0) {
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
    k_dir_pixels<<<blocks, 256, 0, s>>>(d_dirs, n, d_out);
    note_launch();
  }
  return cuda_status(cudaGetLastError());
}

int count4_device(const Graph& g, const FixedW* fw, bool parity, uint64_t* d_even,
                  int64_t* d_odd, double* d_weven, double* d_wodd, const Opts& o, Scratch& sc,
                  bool pix, unsigned long long* weven_out, unsigned long long* wodd_out) {
  cudaStream_t s = o.stream;
  int st = GS_OK;
  pix = pix && parity;
  const uint8_t* pixsign = nullptr;
  if (pix) {
    pixsign = pixel_sign_table(&st);
    if (!pixsign) return st;
  }
  const Conf4Tables* t = conf4_tables(g.nb, &st);
  if (!t) return st;
  const int no = (int)t->n_orbits;
  const bool weighted = fw != nullptr;
  Args a;
  a.ptr = g.d_ptr;
  a.deg = g.d_deg;
  a.adj = nullptr;
  a.adj_off = 0;
  a.split = g.n;
  a.adj_off2 = 0;
  a.big = nullptr;
  a.nbig = 0;
  a.hub_begin = 0;
  a.hub_end = g.n;
  a.xyzp = g.d_xyzp;
  a.e2g = g.d_edges2;
  a.lut = t->d_lut;
  a.n = g.n;
  a.box = g.box_u;
  a.nb = g.nb;
  a.n_orbits = no;
  a.even = reinterpret_cast<unsigned long long*>(d_even);
  a.odd = parity ? (d_odd ? reinterpret_cast<unsigned long long*>(d_odd)
                          : sc.alloc<unsigned long long>(no))
                 : nullptr;
  a.W = weighted ? fw->d_W : nullptr;
  a.pixsign = pixsign;
  a.hub_stride = 1;
  // weighted results land in the callers' 192-bit arrays (or scratch)
  unsigned long long* weven = weighted ? (weven_out ? weven_out : sc.alloc<unsigned long long>(3 * (size_t)no))
                                       : nullptr;
  unsigned long long* wodd = (weighted && parity) ? (wodd_out ? wodd_out : sc.alloc<unsigned long long>(3 * (size_t)no))
                                                  : nullptr;
  a.weven = weven;
  a.wodd = wodd;
  a.hub_counter = sc.alloc<unsigned long long>(2);
  a.err = sc.alloc<int>(1);
  if (!a.hub_counter || !a.err || (parity && !a.odd) || (weighted && !a.weven) ||
      (weighted && parity && !a.wodd))
    return GS_ENOMEM;
  cudaMemsetAsync(a.hub_counter, 0, sizeof(unsigned long long) * 2, s);
  cudaMemsetAsync(a.err, 0, sizeof(int), s);

  int dev = 0, sms = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  // static shared memory: the bucket table, the bin edges and a few words
  const size_t avail = (size_t)optin - 1024 - kBucketMax;
  // bytes of one shared slot: unweighted, the even (and odd) count;
  // weighted, one or three cells of a 128-bit sum and a count
  const size_t per_slot = weighted ? (parity ? 60 : 20) : (parity ? 8 : 4);
  // shared row capacity: the longest row rounded up to 32 (at most
  // kMaxSmemRow), less while the slots do not fit
  int mcap = std::min(kMaxSmemRow, std::max(32, (g.max_deg + 31) & ~31));
  int nh = no;
  // unweighted: every orbit's counts in shared memory when a row capacity of
  // at least 256 leaves room for them; otherwise (and always when weighted)
  // as many slots as fit beside the longest row's workspace
  int mfit = mcap;
  while (!weighted && mfit > 256 && (size_t)no * per_slot + 16 + workspace_bytes(mfit, pix) > avail)
    mfit -= 32;
  if (!weighted && (size_t)no * per_slot + 16 + workspace_bytes(mfit, pix) <= avail) {
    mcap = mfit;
  } else {
    if (workspace_bytes(mcap, pix) + 16 + per_slot > avail) return GS_ERANGE;
    nh = (int)std::min<size_t>((size_t)no, (avail - workspace_bytes(mcap, pix) - 16) / per_slot);
  }
  // variant 8: only 64 shared slots (exercises the global path of the other
  // orbits on any input)
  if (o.variant & 8) nh = std::min(nh, 64);
  // with fewer slots than orbits the orbits are relabelled (most frequent
  // first) and the per-slot results mapped back at the end
  const bool relabel = nh < no;
  unsigned long long* s_even = a.even;
  unsigned long long* s_odd = a.odd;
  unsigned long long* const o_odd = a.odd;  // odd counts in orbit order (caller's or scratch)
  int32_t* d_slot = nullptr;
  uint32_t* d_lut2 = nullptr;
  if (relabel) {
    s_even = sc.alloc<unsigned long long>(no);
    s_odd = parity ? sc.alloc<unsigned long long>(no) : nullptr;
    if (weighted) {
      a.weven = sc.alloc<unsigned long long>(3 * (size_t)no);
      a.wodd = parity ? sc.alloc<unsigned long long>(3 * (size_t)no) : nullptr;
    }
    d_slot = sc.alloc<int32_t>(no);
    d_lut2 = sc.alloc<uint32_t>(t->lut.size());
    if (!s_even || (parity && !s_odd) || (weighted && (!a.weven || (parity && !a.wodd))) ||
        !d_slot || !d_lut2)
      return GS_ENOMEM;
  }
  cudaMemsetAsync(s_even, 0, sizeof(uint64_t) * no, s);
  if (parity) cudaMemsetAsync(s_odd, 0, sizeof(uint64_t) * no, s);
  if (a.weven) cudaMemsetAsync(a.weven, 0, sizeof(unsigned long long) * 3 * no, s);
  if (a.wodd) cudaMemsetAsync(a.wodd, 0, sizeof(unsigned long long) * 3 * no, s);
  a.even = s_even;
  a.odd = s_odd;
  a.hot = nh;

  const bool small_r = g.edges[g.nb] < 32768;
  auto pick = [&](bool P, bool Wt, bool X) -> void (*)(Args) {
#define GS_PICK(P_, Wt_, X_)                                                   \
  return small_r ? k_count4<P_, Wt_, true, X_> : k_count4<P_, Wt_, false, X_>
    if (P && X) {
      if (Wt) GS_PICK(true, true, true);
      GS_PICK(true, false, true);
    }
    if (P) {
      if (Wt) GS_PICK(true, true, false);
      GS_PICK(true, false, false);
    }
    if (Wt) GS_PICK(false, true, false);
    GS_PICK(false, false, false);
#undef GS_PICK
  };
  // variant 1 sends every hub to the global workspace (exercises it on any
  // input)
  const bool force_global = (o.variant & 1) != 0;
  const int thr = force_global ? 2 : mcap;
  void (*kern)(Args) = pick(parity, weighted, pix);
  const size_t smem = (size_t)nh * per_slot + 16 + workspace_bytes(mcap, pix);
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
  const int grid = std::max(1, per_sm) * sms;
  a.mcap = mcap;
  a.thr = thr;
  a.gcap = std::max(g.max_deg, 3);
  // squared-distance buckets no wider than the narrowest bin (variant 4:
  // binary search instead)
  a.bk_shift = 0;
  a.bk_n = 0;
  if (!(o.variant & 4)) {
    int64_t gap = INT64_MAX;
    for (int b = 0; b < g.nb; ++b)
      gap = std::min(gap, g.edges[b + 1] * g.edges[b + 1] - g.edges[b] * g.edges[b]);
    int sh = 0;
    while (sh < 62 && (int64_t(1) << (sh + 1)) <= gap) ++sh;
    const int64_t top = g.edges[g.nb] * g.edges[g.nb];
    const int64_t nbk = ((top - 1) >> sh) + 1;
    if (gap >= 1 && nbk <= kBucketMax) {
      a.bk_shift = sh;
      a.bk_n = (int)nbk;
    }
  }
  a.gscratch = nullptr;
  a.gscratch_stride = 0;
  if (g.max_deg > thr) {
    a.gscratch_stride = (workspace_bytes(a.gcap, pix) + 255) & ~(size_t)255;
    a.gscratch = sc.alloc<unsigned char>(a.gscratch_stride * grid);
    if (!a.gscratch) return GS_ENOMEM;
  }

  // Relabelling: count the tetrahedra of every orbit over an evenly strided
  // sample of about 2048 hubs of the first window (unweighted, all slots in
  // shared memory, long rows skipped), rank the orbits by that count and
  // give the top nh the shared slots. Where that count kernel does not fit,
  // the orbits keep their order. The choice changes only the speed.
  auto relabel_orbits = [&](const Args& wa, cudaStream_t st_) -> int {
    std::vector<int32_t> slot_of(no);
    std::vector<int32_t> order(no);
    for (int k = 0; k < no; ++k) order[k] = k;
    const size_t smem_s = (size_t)no * 4 + 16 + workspace_bytes(mcap, false);
    if (smem_s <= avail) {
      unsigned long long* d_cnt = sc.alloc<unsigned long long>(no);
      unsigned long long* d_hc = sc.alloc<unsigned long long>(1);
      if (!d_cnt || !d_hc) return GS_ENOMEM;
      cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long) * no, st_);
      cudaMemsetAsync(d_hc, 0, sizeof(unsigned long long), st_);
      Args sa = wa;
      sa.big = nullptr;
      sa.nbig = 0;
      sa.thr = mcap;
      sa.hot = no;
      sa.lut = t->d_lut;
      sa.even = d_cnt;
      sa.odd = nullptr;
      sa.weven = sa.wodd = nullptr;
      sa.W = nullptr;
      sa.hub_counter = d_hc;
      sa.hub_stride = std::max<int64_t>(1, (wa.hub_end - wa.hub_begin) / 2048);
      void (*ks)(Args) = pick(false, false, false);
      cudaFuncSetAttribute(ks, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_s);
      int ps = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, ks, kThreads, smem_s);
      ks<<<std::max(1, ps) * sms, kThreads, smem_s, st_>>>(sa);
      note_launch();
      std::vector<unsigned long long> cnt(no);
      cudaMemcpyAsync(cnt.data(), d_cnt, sizeof(unsigned long long) * no, cudaMemcpyDeviceToHost,
                      st_);
      const cudaError_t e = cudaStreamSynchronize(st_);
      if (e != cudaSuccess) return cuda_status(e);
      std::stable_sort(order.begin(), order.end(),
                       [&](int x, int y) { return cnt[x] > cnt[y]; });
    }
    for (int k = 0; k < no; ++k) slot_of[order[k]] = k;
    cudaMemcpyAsync(d_slot, slot_of.data(), sizeof(int32_t) * no, cudaMemcpyHostToDevice, st_);
    const int64_t nl = (int64_t)t->lut.size();
    k_relabel_lut<<<(int)std::min<int64_t>((nl + 255) / 256, 4096), 256, 0, st_>>>(t->d_lut, nl,
                                                                                  d_slot, d_lut2);
    note_launch();
    // the host vector must outlive the (pageable, hence synchronous) copy
    const cudaError_t e = cudaStreamSynchronize(st_);
    return e == cudaSuccess ? cuda_status(cudaGetLastError()) : cuda_status(e);
  };

  KernelTimer timer(o.kernel_ms);
  timer.start(s);
  bool first = true;
  st = for_each_window(g, o, sc, [&](const WinView& v) -> int {
    a.adj = v.adj;
    a.adj_off = v.off1;
    a.split = v.split;
    a.adj_off2 = v.off2;
    a.hub_begin = v.h0;
    a.hub_end = v.h1;
    if (first && relabel) {
      const int rs = relabel_orbits(a, s);
      if (rs) return rs;
      a.lut = d_lut2;
    }
    first = false;
    // the window's long rows go to the front of its hub queue
    std::vector<int64_t> big;
    if (g.max_deg > thr)
      for (int64_t h = v.h0; h < v.h1; ++h)
        if (g.h_deg[h] > thr) big.push_back(h);
    a.nbig = (int64_t)big.size();
    a.big = nullptr;
    if (!big.empty()) {
      int64_t* d_big = sc.alloc<int64_t>(big.size());
      if (!d_big) return GS_ENOMEM;
      cudaMemcpyAsync(d_big, big.data(), sizeof(int64_t) * big.size(), cudaMemcpyHostToDevice, s);
      a.big = d_big;
    }
    cudaMemsetAsync(a.hub_counter, 0, sizeof(unsigned long long), s);
    { kern<<<grid, kThreads, smem, s>>>(a); note_launch(); }
    // the host list must outlive the (pageable, hence synchronous) copy only
    return cuda_status(cudaGetLastError());
  });
  if (st) return st;
  if (relabel) {
    auto back = [&](const unsigned long long* src, int words, unsigned long long* dst) {
      const int64_t n = (int64_t)no * words;
      k_slots_to_orbits<<<(int)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, s>>>(src, d_slot,
                                                                                     no, words, dst);
      note_launch();
    };
    back(s_even, 1, reinterpret_cast<unsigned long long*>(d_even));
    if (parity) back(s_odd, 1, o_odd);
    if (weighted) back(a.weven, 3, weven);
    if (weighted && parity) back(a.wodd, 3, wodd);
  }
  timer.stop(s);
  if (d_weven) {
    if (weighted)
      { k_i192_to_double<<<(no + 255) / 256, 256, 0, s>>>(weven, no, 4 * fw->scale, d_weven); note_launch(); }
    else
      { k_u64_to_double<<<(no + 255) / 256, 256, 0, s>>>(reinterpret_cast<unsigned long long*>(d_even), no, d_weven); note_launch(); }
  }
  if (d_wodd && parity) {
    if (weighted)
      { k_i192_to_double<<<(no + 255) / 256, 256, 0, s>>>(wodd, no, 4 * fw->scale, d_wodd); note_launch(); }
    else
      { k_i64_to_double<<<(no + 255) / 256, 256, 0, s>>>(reinterpret_cast<const long long*>(o_odd), no,
                                                       d_wodd); note_launch(); }
  }
  int herr = 0;
  cudaMemcpyAsync(&herr, a.err, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e);
  timer.publish();
  return herr ? GS_ETIMEOUT : GS_OK;
}

}  // namespace gs
