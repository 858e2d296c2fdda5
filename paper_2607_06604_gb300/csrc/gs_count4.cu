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
  unsigned long long* even;
  unsigned long long* odd;
  unsigned long long* weven;  // [n_orbits][3] 192-bit
  unsigned long long* wodd;
  const int64_t* __restrict__ W;
  const int8_t* __restrict__ pixsign;  // pixelised parity: signs of sorted pixel triples
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
  const int64_t n2 = x * x + y * y + z * z, z64 = 64 * z * z;
  int band = z >= 0 ? 8 : 0;
  for (int s = 1; s <= 7; ++s) {
    const int64_t edge = (int64_t)(s * s) * n2;
    // z >= 0: edges s/8 at or below z/|d|; z < 0: edges -s/8 at or below it
    band += (z >= 0 ? (z64 >= edge) : (z64 <= edge)) ? 1 : 0;
  }
  int sector = 0;
  if (x != 0 || y != 0) {
    // turn by -pi/2 until the direction lies in [0, pi/2): a > 0, b >= 0
    int quarter = 0;
    int64_t a = x, b = y;
    while (!(a > 0 && b >= 0)) {
      const int64_t t = a;
      a = b;
      b = -t;
      ++quarter;
    }
    const int64_t a2 = 2 * a * a;
    int eighth = 0;
    if ((a + b) * (a + b) >= a2) ++eighth;           // phi >= pi/8
    if (b >= a) ++eighth;                            // phi >= pi/4
    if (b > a && (b - a) * (b - a) >= a2) ++eighth;  // phi >= 3pi/8
    sector = 4 * quarter + eighth;
  }
  return 16 * band + sector;
}

// Sign of the pixel volume (u_p1 x u_p2) . u_p3 of three pixel centres: 0
// for repeated pixels, else the table entry of the sorted triple times the
// parity of the sort. The table (host-built in FP64, 0 where |V| < 1e-9) is
// indexed by the combinatorial number C(r,3) + C(q,2) + p of p < q < r.
__device__ inline int pix_sign(const int8_t* __restrict__ T, int p1, int p2, int p3) {
  if (p1 == p2 || p1 == p3 || p2 == p3) return 0;
  int s = 1;
  if (p1 > p2) { const int t = p1; p1 = p2; p2 = t; s = -s; }
  if (p2 > p3) { const int t = p2; p2 = p3; p3 = t; s = -s; }
  if (p1 > p2) { const int t = p1; p1 = p2; p2 = t; s = -s; }
  const int idx = p3 * (p3 - 1) * (p3 - 2) / 6 + p2 * (p2 - 1) / 2 + p1;
  return s * (int)T[idx];
}

struct Workspace {
  uint32_t* row;      // staged N+(i) words
  int4* disp;         // displacement of each neighbour from the hub
  uint32_t* bits;     // m x W bit matrix
  int* cid;           // caller index of each neighbour (pixelised parity)
  uint8_t* brow;      // per warp: bin(a, c) of its current row a, cap bytes each
  uint32_t* queue;    // per-warp queue of (b, c) entries: kWarps x 64 words
  int cap;
};

__device__ inline Workspace carve(unsigned char* p, int cap) {
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
  w.brow = reinterpret_cast<uint8_t*>(p);
  p += (size_t)kWarps * ((cap + 15) & ~15);
  w.queue = reinterpret_cast<uint32_t*>(p);
  w.cap = (cap + 15) & ~15;
  return w;
}

// One hub: stage N+(i), build the neighbour bit matrix, enumerate the
// tetrahedra. GW: the workspace is in global memory (rows above the shared
// capacity) and counts go straight to the global histograms. Returns false
// when the staging copy timed out.
template <bool PARITY, bool WEIGHTED, bool SMALLR, bool GW, bool PIX, class E2T>
__device__ bool hub4(const Args& a, const Workspace& w, const E2T* e2, const uint8_t* bk,
                     unsigned* h_even,
                     int* h_odd, int64_t i, int m, uint64_t* bar, uint32_t& phase, int* s_row) {
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
    w.disp[k] = make_int4((int)mi((int64_t)Q.x - P.x, a.box), (int)mi((int64_t)Q.y - P.y, a.box),
                          (int)mi((int64_t)Q.z - P.z, a.box), (int)edge_bin(row[k]));
    if (PIX) w.cid[k] = Q.w;
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
    const int64_t Wia = WEIGHTED ? Wi * a.W[edge_id(wa)] : 0;
    const uint32_t* bra = w.bits + sa * W;
    // bin(a, c) of every edge (a, c) of the row, once per row: the triangle
    // loop and the drain read b_12 and b_13 from here
    uint8_t* brw = w.brow + (size_t)warp * w.cap;
    for (int c = sa + 1 + lane; c < m; c += 32)
      if ((bra[c >> 5] >> (c & 31)) & 1u)
        brw[c] = (uint8_t)bin_of(d2<SMALLR>(da, w.disp[c]), e2, nb, bk, a.bk_shift);
    __syncwarp();
    int qn = 0;
    // process the first 32 queue entries (or all when draining)
    auto drain = [&](bool all) {
      while (qn >= 32 || (all && qn > 0)) {
        const bool active = lane < qn;
        const uint32_t e = active ? qbc[lane] : 0u;
        __syncwarp();
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
          if (GW) atomicAdd(a.even + orbit, 1ull);
          else atomicAdd(h_even + orbit, 1u);
          long long plo = 0, phi = 0;
          // (W_i W_a)(W_b W_c): two products below 2^60, one 128-bit product
          if (WEIGHTED) {
            mul_i128(Wia, a.W[edge_id(row[sb])] * a.W[edge_id(row[sc])], &plo, &phi);
            atomic_add_i192(a.weven + 3 * orbit, (unsigned long long)plo, (unsigned long long)phi);
          }
          if (PARITY && (ent >> 31)) {
            int sgn;
            if constexpr (PIX) {
              // the pixelised reading: the three spokes from the vertex with
              // the smallest caller index, taken in ascending caller order; a
              // sorting network keeps the displacements (from the hub) and
              // the parity of the reordering
              int key[4] = {P.w, w.cid[sa], w.cid[sb], w.cid[sc]};
              int4 D[4] = {make_int4(0, 0, 0, 0), da, db, dc};
              int par = 1;
              auto cx = [&](int u, int v) {
                if (key[u] > key[v]) {
                  const int tk = key[u];
                  key[u] = key[v];
                  key[v] = tk;
                  const int4 td = D[u];
                  D[u] = D[v];
                  D[v] = td;
                  par = -par;
                }
              };
              cx(0, 1);
              cx(2, 3);
              cx(0, 2);
              cx(1, 3);
              cx(1, 2);
              int px[3];
              bool zero = false;  // coincident points: no direction, degenerate
#pragma unroll
              for (int t = 1; t <= 3; ++t) {
                const int64_t x = (int64_t)D[t].x - D[0].x, y = (int64_t)D[t].y - D[0].y,
                              z = (int64_t)D[t].z - D[0].z;
                zero = zero || (x == 0 && y == 0 && z == 0);
                px[t - 1] = dir_pixel(x, y, z);
              }
              sgn = zero ? 0 : par * pix_sign(a.pixsign, px[0], px[1], px[2]);
            } else {
              const int64_t V = det3<SMALLR>(da, db, dc);
              sgn = V > 0 ? 1 : (V < 0 ? -1 : 0);
            }
            if (sgn != 0) {
              if ((ent >> 30) & 1u) sgn = -sgn;
              if (GW) atomicAdd(a.odd + orbit, (unsigned long long)(long long)sgn);
              else atomicAdd(h_odd + orbit, sgn);
              if (WEIGHTED) {
                unsigned long long lo = (unsigned long long)plo, hi = (unsigned long long)phi;
                if (sgn < 0) {  // negate the 128-bit product
                  lo = ~lo + 1ull;
                  hi = ~hi + (lo == 0ull ? 1ull : 0ull);
                }
                atomic_add_i192(a.wodd + 3 * orbit, lo, hi);
              }
            }
          }
        }
        if (qn >= 32) {  // keep the overflow (the queue holds at most 63)
          const int rest = qn - 32;
          uint32_t mv = 0;
          if (lane < rest) mv = qbc[32 + lane];
          __syncwarp();
          if (lane < rest) qbc[lane] = mv;
          __syncwarp();
          qn = rest;
        } else {
          qn = 0;
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
          if (set) qbc[qn + __popc(x & ((1u << lane) - 1u))] = ((uint32_t)sb << 16) | (uint32_t)(wc * 32 + lane);
          qn += __popc(x);
          __syncwarp();
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
  unsigned* h_even = reinterpret_cast<unsigned*>(smem);
  int* h_odd = reinterpret_cast<int*>(h_even + a.n_orbits);
  unsigned char* sws = smem + (size_t)a.n_orbits * 4 * (PARITY ? 2 : 1);
  sws = reinterpret_cast<unsigned char*>(((uintptr_t)sws + 15) & ~(uintptr_t)15);
  const Workspace ws_s = carve(sws, a.mcap);
  const Workspace ws_g = carve(a.gscratch ? a.gscratch + (size_t)blockIdx.x * a.gscratch_stride
                                          : sws,
                               a.gscratch ? a.gcap : a.mcap);

  for (int k = tid; k < a.n_orbits; k += kThreads) {
    h_even[k] = 0;
    if (PARITY) h_odd[k] = 0;
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
    for (int k = tid; k < a.n_orbits; k += kThreads) {
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
          i = a.hub_begin + qq;
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
    if (m > a.thr)
      ok = hub4<PARITY, WEIGHTED, SMALLR, true, PIX>(a, ws_g, e2, bk, h_even, h_odd, i, m, &bar,
                                                     phase, &s_row);
    else
      ok = hub4<PARITY, WEIGHTED, SMALLR, false, PIX>(a, ws_s, e2, bk, h_even, h_odd, i, m, &bar,
                                                      phase, &s_row);
    if (!ok) return;
  }
  __syncthreads();
  flush();
}

size_t workspace_bytes(int mcap) {
  const size_t Wc = (size_t)(mcap + 31) / 32;
  return (size_t)pad_row(mcap) * 4 + (size_t)mcap * 16 + (size_t)mcap * Wc * 4 +
         (size_t)mcap * 4 + (size_t)kWarps * ((mcap + 15) & ~15) + (size_t)kWarps * 64 * 5 + 64;
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
std::vector<int8_t> g_pix_host;
int8_t* g_pix_dev[64] = {nullptr};

const int8_t* pixel_sign_table(int* status) {
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
    g_pix_host.resize((size_t)256 * 255 * 254 / 6);
    size_t idx = 0;
    for (int r = 0; r < 256; ++r)
      for (int q = 0; q < r; ++q)
        for (int p = 0; p < q; ++p, ++idx) {
          const double* a = u[p];
          const double* b = u[q];
          const double* c = u[r];
          const double v = (a[1] * b[2] - a[2] * b[1]) * c[0] + (a[2] * b[0] - a[0] * b[2]) * c[1] +
                           (a[0] * b[1] - a[1] * b[0]) * c[2];
          g_pix_host[idx] = std::fabs(v) < 1e-9 ? 0 : (v > 0 ? 1 : -1);
        }
  }
  int8_t* d = nullptr;
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
  const int8_t* pixsign = nullptr;
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
  a.weven = weighted ? (weven_out ? weven_out : sc.alloc<unsigned long long>(3 * (size_t)no))
                     : nullptr;
  a.wodd = (weighted && parity) ? (wodd_out ? wodd_out : sc.alloc<unsigned long long>(3 * (size_t)no))
                                : nullptr;
  a.hub_counter = sc.alloc<unsigned long long>(2);
  a.err = sc.alloc<int>(1);
  if (!a.hub_counter || !a.err || (parity && !a.odd) || (weighted && !a.weven) ||
      (weighted && parity && !a.wodd))
    return GS_ENOMEM;
  cudaMemsetAsync(a.even, 0, sizeof(uint64_t) * no, s);
  if (parity) cudaMemsetAsync(a.odd, 0, sizeof(uint64_t) * no, s);
  if (a.weven) cudaMemsetAsync(a.weven, 0, sizeof(unsigned long long) * 3 * no, s);
  if (a.wodd) cudaMemsetAsync(a.wodd, 0, sizeof(unsigned long long) * 3 * no, s);
  cudaMemsetAsync(a.hub_counter, 0, sizeof(unsigned long long) * 2, s);
  cudaMemsetAsync(a.err, 0, sizeof(int), s);

  int dev = 0, sms = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const size_t hist_bytes = (size_t)no * 4 * (parity ? 2 : 1);
  const size_t hist_aligned = (hist_bytes + 15) & ~(size_t)15;
  // largest smem row that fits next to the histograms
  int mcap = kMaxSmemRow;
  // static shared memory: the bucket table, the bin edges and a few words
  const size_t avail = (size_t)optin - 1024 - kBucketMax;
  while (mcap > 32 && hist_aligned + workspace_bytes(mcap) > avail) mcap -= 32;
  if (hist_aligned + workspace_bytes(mcap) > avail) return GS_ERANGE;

  const bool small_r = g.edges[g.nb] < 32768;
  auto pick = [&]() -> void (*)(Args) {
#define GS_PICK(P, Wt, X)                                                    \
  return small_r ? k_count4<P, Wt, true, X> : k_count4<P, Wt, false, X>
    if (parity && pix) {
      if (weighted) GS_PICK(true, true, true);
      GS_PICK(true, false, true);
    }
    if (parity) {
      if (weighted) GS_PICK(true, true, false);
      GS_PICK(true, false, false);
    }
    if (weighted) GS_PICK(false, true, false);
    GS_PICK(false, false, false);
#undef GS_PICK
  };
  // variant 1 sends every hub to the global workspace (exercises it on any
  // input)
  const bool force_global = (o.variant & 1) != 0;
  const int thr = force_global ? 2 : mcap;
  void (*kern)(Args) = pick();
  const size_t smem = hist_aligned + workspace_bytes(mcap);
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
    a.gscratch_stride = (workspace_bytes(a.gcap) + 255) & ~(size_t)255;
    a.gscratch = sc.alloc<unsigned char>(a.gscratch_stride * grid);
    if (!a.gscratch) return GS_ENOMEM;
  }
  KernelTimer timer(o.kernel_ms);
  timer.start(s);
  st = for_each_window(g, o, sc, [&](const WinView& v) -> int {
    a.adj = v.adj;
    a.adj_off = v.off1;
    a.split = v.split;
    a.adj_off2 = v.off2;
    a.hub_begin = v.h0;
    a.hub_end = v.h1;
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
  timer.stop(s);
  if (d_weven) {
    if (weighted)
      { k_i192_to_double<<<(no + 255) / 256, 256, 0, s>>>(a.weven, no, 4 * fw->scale, d_weven); note_launch(); }
    else
      { k_u64_to_double<<<(no + 255) / 256, 256, 0, s>>>(a.even, no, d_weven); note_launch(); }
  }
  if (d_wodd && parity) {
    if (weighted)
      { k_i192_to_double<<<(no + 255) / 256, 256, 0, s>>>(a.wodd, no, 4 * fw->scale, d_wodd); note_launch(); }
    else
      { k_i64_to_double<<<(no + 255) / 256, 256, 0, s>>>(reinterpret_cast<const long long*>(a.odd), no,
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
