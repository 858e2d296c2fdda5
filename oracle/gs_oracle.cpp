// CPU oracle for the binned 3pCF / 4pCF tuple counts of GRAMSCI v2
// (Sabiu, "Fast Graph-based Higher-Order Clustering Statistics on the GPU").
//
// TEST INFRASTRUCTURE ONLY. This file is a plain, slow, obviously correct
// restatement of the paper's definitions. It is used by the test-suite, by
// the smoke check and by the timed CPU baseline of bench.py; the product
// path never links, loads or calls it. It shares no code, header, table or
// helper with the CUDA library.
//
// Definitions implemented (lattice unit u = 1/1024 h^-1 Mpc):
//  * Lattice quantisation: X = floor(1024 x); periodic boxes wrap modulo L_u,
//    open boxes reject coordinates outside [0, L_u).
//  * Displacement i -> j: d = X_j - X_i per axis; in a periodic box of side
//    L_u it is replaced by its minimum image (2d >= L_u: d -= L_u; 2d < -L_u:
//    d += L_u). Squared distance D2 = sum d^2 in 64-bit integers.
//  * Graph (Sec. 2.1, Eq. adjacency): j is a neighbour of i iff j != i and
//    E_0^2 <= D2 < E_nb^2; its radial bin is the largest b with E_b^2 <= D2.
//    Rows are sorted by neighbour index.
//  * Triangle (Sec. 2.2): three points whose three pairs are all edges,
//    counted once; configuration = sorted bin triple, ranked
//    lexicographically (Sec. 5.1).
//  * Tetrahedron (Sec. 2.2): four points whose six pairs are all edges,
//    counted once; configuration = S4 orbit of the labelled edge-bin tuple
//    (b01,b02,b03,b12,b13,b23), represented by its lexicographically
//    smallest member; orbits ranked by representative (Sec. 5.2).
//  * Parity (Sec. 3.2, Eq. volume): V = (r_01 x r_02) . r_03 evaluated in the
//    vertex order that maps the tetrahedron onto its orbit representative.
//    Even channel gets every tetrahedron; the odd channel gets sign(V) when
//    V != 0 and the orbit is chiral (its representative is fixed by no odd
//    permutation, so sign(V) does not depend on the relabelling chosen).
//    Degenerate tetrahedra (V == 0, computed exactly) get zero odd weight.
//  * mu binning (named in the conclusions, not defined): line of sight z;
//    a triangle's mu = |n_z| / |n| for the normal n of its plane; bin =
//    largest m < nmu with m^2 |n|^2 <= nmu^2 n_z^2; collinear: bin nmu.
//  * Pairs and the disconnected term (Sec. 3.3, Eq. disc): pairs[b] counts
//    unordered edges in bin b; xi[b] = pairs[b]/RR[b] - 1; zeta_disc of an
//    orbit = xi(r01)xi(r23) + xi(r02)xi(r13) + xi(r03)xi(r12) on its
//    representative, evaluated left to right in FP64 without contraction.
//
// Algorithms: the graph is built by brute force over all pairs or by a plain
// uniform cell grid with a per-row sort. Triangles are found with the
// two-pointer merge-walk of Sec. 3.1 over the rows restricted to indices
// above the hub; tetrahedra with the three-pointer walk of Eq. (threeway).
// Weighted sums are accumulated exactly: every FP32 weight is an integer
// multiple of a common power of two, products are formed in 128-bit
// integers when they fit and exactly in 256 bits otherwise, summed in a
// 256-bit accumulator, and the exact total is rounded to FP64 once at the
// end, to nearest with ties to even.
//
// Host threads partition hubs; each thread has its own histograms, summed
// at the end (the shape of the paper's OpenMP CPU kernels, Sec. 4.3).

#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

namespace {

typedef __int128 i128;

// ----------------------------------------------------------------------------
// Exact accumulator: a 256-bit two's-complement integer.
struct Acc256 {
  uint64_t w[4] = {0, 0, 0, 0};
  void add(i128 v) {
    uint64_t lo = (uint64_t)v;
    uint64_t hi = (uint64_t)(v >> 64);
    uint64_t ext = (v < 0) ? ~0ull : 0ull;
    uint64_t add_w[4] = {lo, hi, ext, ext};
    unsigned carry = 0;
    for (int k = 0; k < 4; ++k) {
      uint64_t a = w[k];
      uint64_t s = a + add_w[k];
      unsigned c1 = s < a;
      uint64_t s2 = s + carry;
      unsigned c2 = s2 < s;
      w[k] = s2;
      carry = c1 | c2;
    }
  }
  void add(const Acc256& o) {
    unsigned carry = 0;
    for (int k = 0; k < 4; ++k) {
      uint64_t a = w[k];
      uint64_t s = a + o.w[k];
      unsigned c1 = s < a;
      uint64_t s2 = s + carry;
      unsigned c2 = s2 < s;
      w[k] = s2;
      carry = c1 | c2;
    }
  }
  // The exact product a * b of two signed 128-bit integers (below 2^254 in
  // magnitude), as a 256-bit two's-complement value.
  static Acc256 product(i128 a, i128 b) {
    typedef unsigned __int128 u128;
    const bool neg = (a < 0) != (b < 0);
    const u128 ua = a < 0 ? (u128)0 - (u128)a : (u128)a;
    const u128 ub = b < 0 ? (u128)0 - (u128)b : (u128)b;
    const uint64_t a0 = (uint64_t)ua, a1 = (uint64_t)(ua >> 64);
    const uint64_t b0 = (uint64_t)ub, b1 = (uint64_t)(ub >> 64);
    // schoolbook: limb k collects the partial products a_x b_y with x + y = k
    uint64_t limb[4] = {0, 0, 0, 0};
    auto put = [&](int k, u128 v) {
      for (; k < 4 && v; ++k) {
        const u128 t = (u128)limb[k] + (uint64_t)v;
        limb[k] = (uint64_t)t;
        v = (v >> 64) + (t >> 64);
      }
    };
    put(0, (u128)a0 * b0);
    put(1, (u128)a0 * b1);
    put(1, (u128)a1 * b0);
    put(2, (u128)a1 * b1);
    Acc256 r;
    for (int k = 0; k < 4; ++k) r.w[k] = limb[k];
    return neg ? r.negated() : r;
  }
  Acc256 negated() const {
    Acc256 r;
    unsigned carry = 1;
    for (int k = 0; k < 4; ++k) {
      const uint64_t x = ~w[k];
      const uint64_t s2 = x + carry;
      carry = (s2 < x) ? 1u : 0u;
      r.w[k] = s2;
    }
    return r;
  }
  // Bit k of the magnitude m (k outside [0, 256) reads as 0).
  static unsigned bit_of(const uint64_t m[4], int k) {
    if (k < 0 || k >= 256) return 0;
    return (unsigned)((m[k >> 6] >> (k & 63)) & 1ull);
  }
  // Whether any bit of m below index k is set.
  static bool any_below(const uint64_t m[4], int k) {
    for (int q = 0; q < 256 && q < k; ++q)
      if (bit_of(m, q)) return true;
    return false;
  }
  // The value times 2^-scale, rounded to the nearest double with ties to
  // even (IEEE 754 roundTiesToEven), taken straight from the definition:
  // a double keeps the 53 leading bits of a normal number and, below
  // 2^-1022, only the bits worth at least 2^-1074; the kept integer q is
  // raised by one when the first dropped bit is 1 and either a later dropped
  // bit is 1 or q is odd.
  double to_double(int scale) const {
    uint64_t m[4] = {w[0], w[1], w[2], w[3]};
    const bool neg = (m[3] >> 63) != 0;
    if (neg) {  // magnitude of a negative two's-complement value
      unsigned carry = 1;
      for (int k = 0; k < 4; ++k) {
        uint64_t x = ~m[k];
        uint64_t s = x + carry;
        carry = (s < x) ? 1u : 0u;
        m[k] = s;
      }
    }
    int lead = -1;  // index of the leading one bit
    for (int k = 255; k >= 0; --k)
      if (bit_of(m, k)) { lead = k; break; }
    if (lead < 0) return 0.0;
    // index of the last kept bit: 53 significant bits, or the 2^-1074 bit
    // when the value lies below the smallest normal number
    int cut = lead - 52;
    if (lead - scale < -1022) cut = scale - 1074;
    uint64_t q = 0;
    for (int k = lead; k >= cut && k >= 0; --k) q = (q << 1) | bit_of(m, k);
    if (cut > 0) {
      const unsigned half = bit_of(m, cut - 1);
      const bool rest = any_below(m, cut - 1);
      if (half && (rest || (q & 1ull))) q += 1;
    } else {
      cut = 0;  // every bit kept: the value is a double exactly
    }
    const double v = std::ldexp((double)q, cut - scale);  // q <= 2^53: exact
    return neg ? -v : v;
  }
};

// Exact fixed-point weights: W_i = w_i * 2^S is an integer for every i.
struct FixedWeights {
  std::vector<int64_t> W;
  int S = 0;
  int bits = 0;  // max bit length of |W|
  bool ok = true;
};

FixedWeights make_fixed(const float* w, int64_t n) {
  FixedWeights fw;
  fw.W.resize(n);
  int emin = 1 << 30;
  for (int64_t i = 0; i < n; ++i) {
    double x = (double)w[i];
    if (!std::isfinite(x)) { fw.ok = false; return fw; }
    if (x == 0.0) continue;
    int e;
    std::frexp(x, &e);
    emin = std::min(emin, e);
  }
  if (emin == (1 << 30)) emin = 0;
  fw.S = 24 - emin;  // every float with frexp exponent >= emin is k*2^(emin-24)
  for (int64_t i = 0; i < n; ++i) {
    double v = std::ldexp((double)w[i], fw.S);
    if (std::fabs(v) >= 9.0e15 || v != std::trunc(v)) { fw.ok = false; return fw; }
    fw.W[i] = (int64_t)v;
    uint64_t a = (uint64_t)(fw.W[i] < 0 ? -fw.W[i] : fw.W[i]);
    int b = a ? 64 - __builtin_clzll(a) : 0;
    fw.bits = std::max(fw.bits, b);
  }
  return fw;
}

// ----------------------------------------------------------------------------
struct Graph {
  int64_t n = 0;
  int64_t box_u = 0;  // 0 = open box
  int nb = 0;
  std::vector<int64_t> edges;   // nb+1 lattice-unit bin edges
  std::vector<int64_t> edges2;  // squared
  std::vector<int32_t> xyz;     // 3n
  std::vector<int64_t> ptr;     // n+1, full (both directions) adjacency
  std::vector<int32_t> nbr;
  std::vector<uint8_t> bin;
};

inline int64_t min_image(int64_t d, int64_t box) {
  if (box > 0) {
    if (2 * d >= box) d -= box;
    else if (2 * d < -box) d += box;
  }
  return d;
}

inline void displacement(const Graph& g, int64_t i, int64_t j, int64_t d[3]) {
  for (int a = 0; a < 3; ++a)
    d[a] = min_image((int64_t)g.xyz[3 * j + a] - (int64_t)g.xyz[3 * i + a], g.box_u);
}

inline int64_t dist2(const Graph& g, int64_t i, int64_t j) {
  int64_t d[3];
  displacement(g, i, j, d);
  return d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
}

// Bin of a squared distance, or -1 when it is not an edge.
inline int bin_of(const Graph& g, int64_t D2) {
  if (D2 < g.edges2[0] || D2 >= g.edges2[g.nb]) return -1;
  int b = 0;
  while (b + 1 < g.nb && g.edges2[b + 1] <= D2) ++b;
  return b;
}

template <class F>
void parallel_for(int64_t n, int nthreads, F f) {
  if (nthreads <= 1 || n < 64) {
    for (int64_t i = 0; i < n; ++i) f(i, 0);
    return;
  }
  std::atomic<int64_t> next(0);
  const int64_t chunk = 16;
  std::vector<std::thread> th;
  for (int t = 0; t < nthreads; ++t)
    th.emplace_back([&, t]() {
      for (;;) {
        int64_t s = next.fetch_add(chunk);
        if (s >= n) break;
        int64_t e = std::min(n, s + chunk);
        for (int64_t i = s; i < e; ++i) f(i, t);
      }
    });
  for (auto& x : th) x.join();
}

void finish_rows(Graph& g, std::vector<std::vector<std::pair<int32_t, uint8_t>>>& rows) {
  g.ptr.assign(g.n + 1, 0);
  for (int64_t i = 0; i < g.n; ++i) g.ptr[i + 1] = g.ptr[i] + (int64_t)rows[i].size();
  g.nbr.resize(g.ptr[g.n]);
  g.bin.resize(g.ptr[g.n]);
  for (int64_t i = 0; i < g.n; ++i) {
    auto& r = rows[i];
    std::sort(r.begin(), r.end());
    for (size_t k = 0; k < r.size(); ++k) {
      g.nbr[g.ptr[i] + k] = r[k].first;
      g.bin[g.ptr[i] + k] = r[k].second;
    }
    std::vector<std::pair<int32_t, uint8_t>>().swap(r);
  }
}

void build_bruteforce(Graph& g, int nthreads) {
  std::vector<std::vector<std::pair<int32_t, uint8_t>>> rows(g.n);
  parallel_for(g.n, nthreads, [&](int64_t i, int) {
    for (int64_t j = 0; j < g.n; ++j) {
      if (j == i) continue;
      int b = bin_of(g, dist2(g, i, j));
      if (b >= 0) rows[i].push_back({(int32_t)j, (uint8_t)b});
    }
  });
  finish_rows(g, rows);
}

void build_grid(Graph& g, int nthreads) {
  const int64_t rmax = g.edges[g.nb];
  int64_t nc[3], lo[3], width[3];
  for (int a = 0; a < 3; ++a) {
    if (g.box_u > 0) {
      lo[a] = 0;
      nc[a] = std::max<int64_t>(1, std::min<int64_t>(g.box_u / rmax, 256));
      width[a] = 0;  // periodic cells: c = X * nc / box
    } else {
      int64_t mn = INT64_MAX, mx = INT64_MIN;
      for (int64_t i = 0; i < g.n; ++i) {
        mn = std::min<int64_t>(mn, g.xyz[3 * i + a]);
        mx = std::max<int64_t>(mx, g.xyz[3 * i + a]);
      }
      if (g.n == 0) mn = mx = 0;
      lo[a] = mn;
      width[a] = std::max<int64_t>(rmax, (mx - mn) / 256 + 1);
      nc[a] = (mx - mn) / width[a] + 1;
    }
  }
  auto cell_of = [&](int64_t i, int a) -> int64_t {
    int64_t X = g.xyz[3 * i + a];
    if (g.box_u > 0) return X * nc[a] / g.box_u;
    return (X - lo[a]) / width[a];
  };
  const int64_t ncell = nc[0] * nc[1] * nc[2];
  std::vector<std::vector<int32_t>> cells(ncell);
  for (int64_t i = 0; i < g.n; ++i) {
    int64_t c = (cell_of(i, 0) * nc[1] + cell_of(i, 1)) * nc[2] + cell_of(i, 2);
    cells[c].push_back((int32_t)i);
  }
  std::vector<std::vector<std::pair<int32_t, uint8_t>>> rows(g.n);
  parallel_for(g.n, nthreads, [&](int64_t i, int) {
    int64_t ci[3] = {cell_of(i, 0), cell_of(i, 1), cell_of(i, 2)};
    std::vector<int64_t> visit;
    for (int dx = -1; dx <= 1; ++dx)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dz = -1; dz <= 1; ++dz) {
          int64_t c[3] = {ci[0] + dx, ci[1] + dy, ci[2] + dz};
          bool skip = false;
          for (int a = 0; a < 3; ++a) {
            if (g.box_u > 0) c[a] = ((c[a] % nc[a]) + nc[a]) % nc[a];
            else if (c[a] < 0 || c[a] >= nc[a]) skip = true;
          }
          if (skip) continue;
          visit.push_back((c[0] * nc[1] + c[1]) * nc[2] + c[2]);
        }
    std::sort(visit.begin(), visit.end());
    visit.erase(std::unique(visit.begin(), visit.end()), visit.end());
    for (int64_t c : visit)
      for (int32_t j : cells[c]) {
        if (j == i) continue;
        int b = bin_of(g, dist2(g, i, j));
        if (b >= 0) rows[i].push_back({j, (uint8_t)b});
      }
  });
  finish_rows(g, rows);
}

// Suffix of row i holding the neighbours with index > i (the rows are sorted).
inline int64_t upper_start(const Graph& g, int64_t i) {
  const int32_t* b = g.nbr.data() + g.ptr[i];
  const int32_t* e = g.nbr.data() + g.ptr[i + 1];
  return g.ptr[i] + (std::upper_bound(b, e, (int32_t)i) - b);
}

// ----------------------------------------------------------------------------
// Configuration enumeration.

// Rank of a sorted triple a <= b <= c among all sorted triples over [0, nb),
// in lexicographic order, via an explicit table.
struct Conf3 {
  int nb;
  std::vector<int32_t> rank;  // nb^3 (indexed by the sorted triple)
  std::vector<std::array<uint8_t, 3>> reps;
  explicit Conf3(int nb_) : nb(nb_), rank((size_t)nb_ * nb_ * nb_, -1) {
    for (int a = 0; a < nb; ++a)
      for (int b = a; b < nb; ++b)
        for (int c = b; c < nb; ++c) {
          rank[((size_t)a * nb + b) * nb + c] = (int32_t)reps.size();
          reps.push_back({(uint8_t)a, (uint8_t)b, (uint8_t)c});
        }
  }
  int of(int x, int y, int z) const {
    int v[3] = {x, y, z};
    std::sort(v, v + 3);
    return rank[((size_t)v[0] * nb + v[1]) * nb + v[2]];
  }
};

// Edge slot of the vertex pair (a, b) in the tuple (01, 02, 03, 12, 13, 23).
inline int edge_slot(int a, int b) {
  if (a > b) std::swap(a, b);
  static const int slot[4][4] = {{-1, 0, 1, 2}, {0, -1, 3, 4}, {1, 3, -1, 5}, {2, 4, 5, -1}};
  return slot[a][b];
}

struct Perm4 {
  int p[4];
  int sign;
};

std::vector<Perm4> all_perms() {
  std::vector<Perm4> out;
  int p[4] = {0, 1, 2, 3};
  do {
    Perm4 q;
    int inv = 0;
    for (int a = 0; a < 4; ++a) {
      q.p[a] = p[a];
      for (int b = a + 1; b < 4; ++b) inv += p[a] > p[b];
    }
    q.sign = (inv % 2) ? -1 : 1;
    out.push_back(q);
  } while (std::next_permutation(p, p + 4));
  return out;
}

typedef std::array<uint8_t, 6> Tup6;

// Relabelled tuple: new vertex k is old vertex pi(k), so the new edge (a, b)
// carries the bin of the old edge (pi(a), pi(b)).
inline Tup6 relabel(const Tup6& t, const Perm4& pi) {
  Tup6 r;
  for (int a = 0; a < 4; ++a)
    for (int b = a + 1; b < 4; ++b) r[edge_slot(a, b)] = t[edge_slot(pi.p[a], pi.p[b])];
  return r;
}

struct Conf4 {
  int nb;
  std::vector<Perm4> perms;
  std::vector<int32_t> orbit;  // nb^6, orbit rank of each raw tuple
  std::vector<uint8_t> perm;   // index of a permutation mapping the raw tuple to its rep
  std::vector<Tup6> reps;
  std::vector<uint8_t> chiral;  // per orbit
  explicit Conf4(int nb_) : nb(nb_) {
    perms = all_perms();
    size_t total = 1;
    for (int k = 0; k < 6; ++k) total *= (size_t)nb;
    orbit.assign(total, -1);
    perm.assign(total, 0);
    std::vector<size_t> rep_index(total);
    // pass 1: representative of every raw tuple
    for (size_t idx = 0; idx < total; ++idx) {
      Tup6 t = decode(idx);
      Tup6 best = t;
      int bestp = 0;
      for (int q = 0; q < 24; ++q) {
        Tup6 r = relabel(t, perms[q]);
        if (r < best) { best = r; bestp = q; }
      }
      // bestp stays the identity (index 0) when t is its own representative
      if (best == t) bestp = 0;
      perm[idx] = (uint8_t)bestp;
      rep_index[idx] = encode(best);
    }
    // pass 2: orbits ranked by representative in lexicographic order; the
    // encoding is lexicographic, so scanning indices in order ranks them.
    std::vector<int32_t> rank_of(total, -1);
    for (size_t idx = 0; idx < total; ++idx)
      if (rep_index[idx] == idx) {
        rank_of[idx] = (int32_t)reps.size();
        reps.push_back(decode(idx));
      }
    for (size_t idx = 0; idx < total; ++idx) orbit[idx] = rank_of[rep_index[idx]];
    chiral.assign(reps.size(), 1);
    for (size_t o = 0; o < reps.size(); ++o)
      for (int q = 0; q < 24; ++q)
        if (perms[q].sign < 0 && relabel(reps[o], perms[q]) == reps[o]) chiral[o] = 0;
  }
  Tup6 decode(size_t idx) const {
    Tup6 t;
    for (int k = 5; k >= 0; --k) {
      t[k] = (uint8_t)(idx % nb);
      idx /= nb;
    }
    return t;
  }
  size_t encode(const Tup6& t) const {
    size_t idx = 0;
    for (int k = 0; k < 6; ++k) idx = idx * nb + t[k];
    return idx;
  }
};

// ----------------------------------------------------------------------------
// Direction pixels for the pixelised parity channel (Sec. 3.2: each spoke's
// direction is quantised to a pixel on the unit sphere, one byte per edge;
// tetrahedra whose pixel volume is below 1e-9 in magnitude are degenerate).
// The paper does not fix the pixel scheme; the reading taken here is 256
// equal-area pixels: 16 bands of equal width in z = cos(theta) times 16
// sectors of equal width in the azimuth phi, pixel = 16 * band + sector.
// Band and sector of an integer direction are decided exactly in integers:
//   band   = number of k in 1..15 with z / |d| >= -1 + k / 8;
//   sector = floor(phi / (pi / 8)), phi = atan2(y, x) in [0, 2 pi), and
//            sector 0 for a direction along the z axis.
// The pixel centre is z_c = -1 + (band + 1/2) / 8, phi_c = (sector + 1/2) pi / 8.

// Whether z / |d| >= s / 8 for s in -7..7, with n2 = |d|^2 (exact).
bool z_at_least(int64_t z, int64_t n2, int s) {
  const int64_t lhs = 64 * z * z, rhs = (int64_t)s * s * n2;
  if (s <= 0) return z >= 0 || lhs <= rhs;
  return z > 0 && lhs >= rhs;
}

int direction_pixel(int64_t x, int64_t y, int64_t z) {
  const int64_t n2 = x * x + y * y + z * z;
  int band = 0;
  for (int k = 1; k <= 15; ++k)
    if (z_at_least(z, n2, k - 8)) ++band;
  int sector = 0;
  if (x != 0 || y != 0) {
    // rotate by a multiple of pi/2 into a > 0, b >= 0 (theta in [0, pi/2))
    int quadrant;
    int64_t a, b;
    if (x > 0 && y >= 0) { quadrant = 0; a = x; b = y; }
    else if (x <= 0 && y > 0) { quadrant = 1; a = y; b = -x; }
    else if (x < 0 && y <= 0) { quadrant = 2; a = -x; b = -y; }
    else { quadrant = 3; a = -y; b = x; }
    // theta >= pi/8  <=>  b >= (sqrt2 - 1) a  <=>  (a + b)^2 >= 2 a^2
    // theta >= pi/4  <=>  b >= a
    // theta >= 3pi/8 <=>  b >= (sqrt2 + 1) a  <=>  b > a and (b - a)^2 >= 2 a^2
    int sub = 0;
    if ((a + b) * (a + b) >= 2 * a * a) ++sub;
    if (b >= a) ++sub;
    if (b > a && (b - a) * (b - a) >= 2 * a * a) ++sub;
    sector = 4 * quadrant + sub;
  }
  return 16 * band + sector;
}

void pixel_centre(int p, double u[3]) {
  const int band = p / 16, sector = p % 16;
  const double zc = -1.0 + (band + 0.5) / 8.0;
  const double phi = (sector + 0.5) * M_PI / 8.0;
  const double rho = std::sqrt(1.0 - zc * zc);
  u[0] = rho * std::cos(phi);
  u[1] = rho * std::sin(phi);
  u[2] = zc;
}

// (u1 x u2) . u3 of three pixel centres, FP64, left to right (no contraction:
// the file is compiled with -ffp-contract=off).
double pixel_volume(int p1, int p2, int p3) {
  double a[3], b[3], c[3];
  pixel_centre(p1, a);
  pixel_centre(p2, b);
  pixel_centre(p3, c);
  const double cx = a[1] * b[2] - a[2] * b[1];
  const double cy = a[2] * b[0] - a[0] * b[2];
  const double cz = a[0] * b[1] - a[1] * b[0];
  return cx * c[0] + cy * c[1] + cz * c[2];
}

constexpr double kDegenerateVolume = 1e-9;

Conf4* conf4_cached(int nb) {
  static std::map<int, Conf4*> cache;
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(nb);
  if (it != cache.end()) return it->second;
  Conf4* c = new Conf4(nb);
  cache[nb] = c;
  return c;
}

}  // namespace

// ============================================================================
extern "C" {

// Conversion of an exact 256-bit two's-complement integer (four 64-bit words,
// least significant first) times 2^-scale to double, exposed for the pins of
// the final rounding step.
double or_exact_to_double(const uint64_t* words, int scale) {
  Acc256 a;
  for (int k = 0; k < 4; ++k) a.w[k] = words[k];
  return a.to_double(scale);
}

// Sec. 2.1 input: float positions (h^-1 Mpc) -> int32 lattice coordinates.
// Returns 0, or -1 when an open-box coordinate falls outside [0, box_u).
int or_quantize(const double* pos, int64_t n, int64_t box_u, int periodic, int32_t* out) {
  for (int64_t i = 0; i < 3 * n; ++i) {
    int64_t X = (int64_t)std::floor(pos[i] * 1024.0);
    if (periodic) {
      X %= box_u;
      if (X < 0) X += box_u;
    } else if (X < 0 || X >= box_u) {
      return -1;
    }
    out[i] = (int32_t)X;
  }
  return 0;
}

// Builds the full sorted adjacency (Sec. 2.1). method 0 = all pairs, 1 = grid.
void* or_graph_build(const int32_t* xyz, int64_t n, int64_t box_u, const int64_t* edges_u,
                     int nb, int method, int nthreads) {
  Graph* g = new Graph();
  g->n = n;
  g->box_u = box_u;
  g->nb = nb;
  g->edges.assign(edges_u, edges_u + nb + 1);
  g->edges2.resize(nb + 1);
  for (int b = 0; b <= nb; ++b) g->edges2[b] = edges_u[b] * edges_u[b];
  g->xyz.assign(xyz, xyz + 3 * n);
  if (method == 0) build_bruteforce(*g, nthreads);
  else build_grid(*g, nthreads);
  return g;
}

int64_t or_graph_num_edges(void* gp) { return ((Graph*)gp)->ptr.back(); }

void or_graph_export(void* gp, int64_t* ptr, int32_t* nbr, uint8_t* bin) {
  Graph* g = (Graph*)gp;
  std::memcpy(ptr, g->ptr.data(), sizeof(int64_t) * (g->n + 1));
  std::memcpy(nbr, g->nbr.data(), sizeof(int32_t) * g->nbr.size());
  std::memcpy(bin, g->bin.data(), g->bin.size());
}

void or_graph_free(void* gp) { delete (Graph*)gp; }

int64_t or_num_configs(int npoint, int nb) {
  if (npoint == 3) return (int64_t)Conf3(nb).reps.size();
  if (npoint == 4) return (int64_t)conf4_cached(nb)->reps.size();
  return -1;
}

int or_config_bins(int npoint, int nb, int64_t idx, uint8_t* bins, int* chiral) {
  if (npoint == 3) {
    Conf3 c(nb);
    if (idx < 0 || idx >= (int64_t)c.reps.size()) return -1;
    for (int k = 0; k < 3; ++k) bins[k] = c.reps[idx][k];
    if (chiral) *chiral = 0;
    return 0;
  }
  if (npoint == 4) {
    Conf4* c = conf4_cached(nb);
    if (idx < 0 || idx >= (int64_t)c->reps.size()) return -1;
    for (int k = 0; k < 6; ++k) bins[k] = c->reps[idx][k];
    if (chiral) *chiral = c->chiral[idx];
    return 0;
  }
  return -1;
}

// Sec. 2.2 / Sec. 3.1: triangles with hub in [hub_lo, hub_hi), each counted at
// its smallest vertex. counts: C(nb+2,3) u64; wsum: NULL or C(nb+2,3) FP64.
// Returns 0, or -2 when the weights cannot be summed exactly.
int or_count_3pcf(void* gp, const float* w, uint64_t* counts, double* wsum, int64_t hub_lo,
                  int64_t hub_hi, int nthreads) {
  Graph& g = *(Graph*)gp;
  Conf3 conf(g.nb);
  const size_t nconf = conf.reps.size();
  FixedWeights fw;
  if (w) {
    fw = make_fixed(w, g.n);
    // |W| < 2^53: W_i W_j fits 128 bits; the triple product is formed in
    // 128 bits when it fits, else exactly in 256 bits
    if (!fw.ok || fw.bits > 53) return -2;
  }
  if (hub_hi < 0 || hub_hi > g.n) hub_hi = g.n;
  if (hub_lo < 0) hub_lo = 0;
  const int nt = std::max(1, nthreads);
  const bool narrow = 3 * (fw.bits + 1) <= 126;
  std::vector<std::vector<uint64_t>> hc(nt, std::vector<uint64_t>(nconf, 0));
  std::vector<std::vector<Acc256>> hw(w ? nt : 0, std::vector<Acc256>(nconf));
  parallel_for(std::max<int64_t>(0, hub_hi - hub_lo), nt, [&](int64_t t, int tid) {
    const int64_t i = hub_lo + t;
    const int64_t s_i = upper_start(g, i), e_i = g.ptr[i + 1];
    for (int64_t p = s_i; p < e_i; ++p) {
      const int32_t j = g.nbr[p];
      const int b_ij = g.bin[p];
      // a walks the hub tail after j; b walks N+(j)
      int64_t a = p + 1, b = upper_start(g, j);
      const int64_t e_j = g.ptr[j + 1];
      while (a < e_i && b < e_j) {
        const int32_t ka = g.nbr[a], kb = g.nbr[b];
        if (ka == kb) {
          const int c = conf.of(b_ij, g.bin[a], g.bin[b]);
          hc[tid][c] += 1;
          if (w) {
            if (narrow) hw[tid][c].add((i128)fw.W[i] * fw.W[j] * fw.W[ka]);
            else hw[tid][c].add(Acc256::product((i128)fw.W[i] * fw.W[j], (i128)fw.W[ka]));
          }
          ++a;
          ++b;
        } else if (ka < kb) {
          ++a;
        } else {
          ++b;
        }
      }
    }
  });
  for (size_t c = 0; c < nconf; ++c) {
    uint64_t s = 0;
    Acc256 acc;
    for (int t = 0; t < nt; ++t) {
      s += hc[t][c];
      if (w) acc.add(hw[t][c]);
    }
    counts[c] = s;
    if (wsum) wsum[c] = w ? acc.to_double(3 * fw.S) : (double)s;
  }
  return 0;
}

// Anisotropic 3pCF (the paper's conclusions name mu binning for
// redshift-space distortions without defining it; this is the reading used
// here). Line of sight: the z axis (distant observer). A triangle's mu is
// |n_z| / |n| for the normal n = d_ij x d_ik of its plane (d the
// minimum-image displacements from the hub), which no relabelling of the
// vertices changes. mu bin m in [0, nmu): the largest m with m / nmu <= mu,
// i.e. m^2 |n|^2 <= nmu^2 n_z^2 in exact integers (mu = 1 falls in the last
// bin); collinear triangles (n = 0) go to the extra bin nmu.
// counts / wsum: [C(nb+2,3)][nmu + 1]. Returns 0, -1 for nmu outside
// [1, 64] or E_nb >= 2^27, -2 when the weights cannot be summed exactly.
int or_count_3pcf_mu(void* gp, const float* w, int nmu, uint64_t* counts, double* wsum,
                     int nthreads) {
  Graph& g = *(Graph*)gp;
  if (nmu < 1 || nmu > 64) return -1;
  // E_nb < 2^27 keeps every product below in 128 bits
  if (g.edges2[g.nb] >= ((int64_t)1 << 54)) return -1;
  Conf3 conf(g.nb);
  const size_t nconf = conf.reps.size();
  const size_t ncell = nconf * (size_t)(nmu + 1);
  FixedWeights fw;
  if (w) {
    fw = make_fixed(w, g.n);
    if (!fw.ok || fw.bits > 53) return -2;
  }
  const int nt = std::max(1, nthreads);
  const bool narrow = 3 * (fw.bits + 1) <= 126;
  std::vector<std::vector<uint64_t>> hc(nt, std::vector<uint64_t>(ncell, 0));
  std::vector<std::vector<Acc256>> hw(w ? nt : 0, std::vector<Acc256>(ncell));
  parallel_for(g.n, nt, [&](int64_t i, int tid) {
    const int64_t s_i = upper_start(g, i), e_i = g.ptr[i + 1];
    for (int64_t p = s_i; p < e_i; ++p) {
      const int32_t j = g.nbr[p];
      const int b_ij = g.bin[p];
      int64_t a = p + 1, b = upper_start(g, j);
      const int64_t e_j = g.ptr[j + 1];
      while (a < e_i && b < e_j) {
        const int32_t ka = g.nbr[a], kb = g.nbr[b];
        if (ka == kb) {
          int64_t u[3], v[3];
          displacement(g, i, j, u);
          displacement(g, i, ka, v);
          const i128 nx = (i128)u[1] * v[2] - (i128)u[2] * v[1];
          const i128 ny = (i128)u[2] * v[0] - (i128)u[0] * v[2];
          const i128 nz = (i128)u[0] * v[1] - (i128)u[1] * v[0];
          const i128 n2 = nx * nx + ny * ny + nz * nz;
          int m = nmu;  // collinear
          if (n2 != 0) {
            m = nmu - 1;
            while (m > 0 && (i128)m * m * n2 > (i128)nmu * nmu * (nz * nz)) --m;
          }
          const size_t c = (size_t)conf.of(b_ij, g.bin[a], g.bin[b]) * (nmu + 1) + m;
          hc[tid][c] += 1;
          if (w) {
            const i128 wij = (i128)fw.W[i] * fw.W[j];
            if (narrow) hw[tid][c].add(wij * fw.W[ka]);
            else hw[tid][c].add(Acc256::product(wij, (i128)fw.W[ka]));
          }
          ++a;
          ++b;
        } else if (ka < kb) {
          ++a;
        } else {
          ++b;
        }
      }
    }
  });
  for (size_t c = 0; c < ncell; ++c) {
    uint64_t s = 0;
    Acc256 acc;
    for (int t = 0; t < nt; ++t) {
      s += hc[t][c];
      if (w) acc.add(hw[t][c]);
    }
    counts[c] = s;
    if (wsum) wsum[c] = w ? acc.to_double(3 * fw.S) : (double)s;
  }
  return 0;
}

// Sec. 2.2, Eq. (threeway), Sec. 3.2: tetrahedra i < j1 < j2 < j3 found at
// hub i; even/odd channels. Any output pointer may be NULL.
// pixel != 0: the odd channel takes the sign of the pixel volume of the
// hub's three spokes (the hub has the smallest index, j1 < j2 < j3), times
// the parity of the relabelling onto the orbit representative, and nothing
// when that volume is below 1e-9 in magnitude (the pixelised reading of
// Sec. 3.2); otherwise the exact integer V in the representative's order.
static int count_4pcf(void* gp, const float* w, uint64_t* even, int64_t* odd, double* weven,
                      double* wodd, int nthreads, int pixel) {
  Graph& g = *(Graph*)gp;
  Conf4* conf = conf4_cached(g.nb);
  const size_t nconf = conf->reps.size();
  FixedWeights fw;
  if (w) {
    fw = make_fixed(w, g.n);
    // |W| < 2^52: a product of four weights and the sum of up to 2^46 of
    // them stay inside the 256-bit accumulator
    if (!fw.ok || fw.bits > 52) return -2;
  }
  const int nt = std::max(1, nthreads);
  std::vector<std::vector<uint64_t>> he(nt, std::vector<uint64_t>(nconf, 0));
  std::vector<std::vector<int64_t>> ho(nt, std::vector<int64_t>(nconf, 0));
  std::vector<std::vector<Acc256>> hwe(w ? nt : 0, std::vector<Acc256>(nconf));
  std::vector<std::vector<Acc256>> hwo(w ? nt : 0, std::vector<Acc256>(nconf));
  parallel_for(g.n, nt, [&](int64_t i, int tid) {
    const int64_t s_i = upper_start(g, i), e_i = g.ptr[i + 1];
    for (int64_t p1 = s_i; p1 < e_i; ++p1) {
      const int32_t j1 = g.nbr[p1];
      const int64_t s_j1 = upper_start(g, j1), e_j1 = g.ptr[j1 + 1];
      // k2 walk: j2 in (hub tail after j1) and in N+(j1)
      int64_t a = p1 + 1, b = s_j1;
      while (a < e_i && b < e_j1) {
        const int32_t ka = g.nbr[a], kb = g.nbr[b];
        if (ka < kb) { ++a; continue; }
        if (kb < ka) { ++b; continue; }
        const int32_t j2 = ka;
        const int64_t p2 = a, q12 = b;
        // three-way walk for j3: alpha over the hub tail after j2, beta over
        // N(j1) after j2, gamma over N(j2) after j2.
        int64_t al = p2 + 1, be = q12 + 1, ga = upper_start(g, j2);
        const int64_t e_j2 = g.ptr[j2 + 1];
        while (al < e_i && be < e_j1 && ga < e_j2) {
          const int32_t ha = g.nbr[al], hb = g.nbr[be], hg = g.nbr[ga];
          if (ha == hb && hb == hg) {
            const int32_t j3 = ha;
            Tup6 t = {g.bin[p1], g.bin[p2], g.bin[al], g.bin[q12], g.bin[be], g.bin[ga]};
            const size_t raw = conf->encode(t);
            const int o = conf->orbit[raw];
            he[tid][o] += 1;
            Acc256 prod;
            if (w) {
              prod = Acc256::product((i128)fw.W[i] * fw.W[j1], (i128)fw.W[j2] * fw.W[j3]);
              hwe[tid][o].add(prod);
            }
            if (conf->chiral[o]) {
              // vertices in the order that maps the tuple onto the representative
              const int64_t v[4] = {i, j1, j2, j3};
              const Perm4& pi = conf->perms[conf->perm[raw]];
              int s = 0;
              if (pixel) {
                // a spoke of zero length (coincident points) has no direction:
                // the tetrahedron is degenerate
                int px[3];
                bool zero = false;
                const int64_t u[3] = {j1, j2, j3};
                for (int k = 0; k < 3; ++k) {
                  int64_t d[3];
                  displacement(g, i, u[k], d);
                  zero = zero || (d[0] == 0 && d[1] == 0 && d[2] == 0);
                  px[k] = direction_pixel(d[0], d[1], d[2]);
                }
                const double Vp = zero ? 0.0 : pixel_volume(px[0], px[1], px[2]);
                if (std::fabs(Vp) >= kDegenerateVolume) s = (Vp > 0 ? 1 : -1) * pi.sign;
              } else {
                int64_t d[3][3];
                for (int k = 1; k <= 3; ++k) displacement(g, v[pi.p[0]], v[pi.p[k]], d[k - 1]);
                const i128 V =
                    (i128)d[0][0] * ((i128)d[1][1] * d[2][2] - (i128)d[1][2] * d[2][1]) -
                    (i128)d[0][1] * ((i128)d[1][0] * d[2][2] - (i128)d[1][2] * d[2][0]) +
                    (i128)d[0][2] * ((i128)d[1][0] * d[2][1] - (i128)d[1][1] * d[2][0]);
                if (V != 0) s = V > 0 ? 1 : -1;
              }
              if (s != 0) {
                ho[tid][o] += s;
                if (w) hwo[tid][o].add(s > 0 ? prod : prod.negated());
              }
            }
            ++al;
            ++be;
            ++ga;
          } else {
            const int32_t mn = std::min(ha, std::min(hb, hg));
            if (ha == mn) ++al;
            if (hb == mn) ++be;
            if (hg == mn) ++ga;
          }
        }
        ++a;
        ++b;
      }
    }
  });
  for (size_t c = 0; c < nconf; ++c) {
    uint64_t se = 0;
    int64_t so = 0;
    Acc256 ae, ao;
    for (int t = 0; t < nt; ++t) {
      se += he[t][c];
      so += ho[t][c];
      if (w) { ae.add(hwe[t][c]); ao.add(hwo[t][c]); }
    }
    if (even) even[c] = se;
    if (odd) odd[c] = so;
    if (weven) weven[c] = w ? ae.to_double(4 * fw.S) : (double)se;
    if (wodd) wodd[c] = w ? ao.to_double(4 * fw.S) : (double)so;
  }
  return 0;
}

int or_count_4pcf(void* gp, const float* w, uint64_t* even, int64_t* odd, double* weven,
                  double* wodd, int nthreads) {
  return count_4pcf(gp, w, even, odd, weven, wodd, nthreads, 0);
}

// Sec. 3.2 with pixelised directions (the reading described at
// direction_pixel): even channel as or_count_4pcf, odd channel from the
// sign of the pixel volume, degenerate tetrahedra (|V| < 1e-9) excluded.
int or_count_4pcf_pix(void* gp, const float* w, uint64_t* even, int64_t* odd, double* weven,
                      double* wodd, int nthreads) {
  return count_4pcf(gp, w, even, odd, weven, wodd, nthreads, 1);
}

// Test hooks: the pixel of integer directions (n of them, [n][3]) and the
// pixel volume of pixel triples ([n][3]).
void or_direction_pixels(const int64_t* d, int64_t n, uint8_t* pix) {
  for (int64_t k = 0; k < n; ++k) pix[k] = (uint8_t)direction_pixel(d[3 * k], d[3 * k + 1], d[3 * k + 2]);
}
void or_pixel_volumes(const int32_t* p, int64_t n, double* v) {
  for (int64_t k = 0; k < n; ++k) v[k] = pixel_volume(p[3 * k], p[3 * k + 1], p[3 * k + 2]);
}

// Sec. 3.3: pair histogram over unordered edges; weighted sums exact.
int or_pairs(void* gp, const float* w, uint64_t* pairs, double* wpairs) {
  Graph& g = *(Graph*)gp;
  FixedWeights fw;
  if (w) {
    fw = make_fixed(w, g.n);
    if (!fw.ok) return -2;
  }
  std::vector<uint64_t> c(g.nb, 0);
  std::vector<Acc256> a(g.nb);
  for (int64_t i = 0; i < g.n; ++i)
    for (int64_t p = upper_start(g, i); p < g.ptr[i + 1]; ++p) {
      c[g.bin[p]] += 1;
      if (w) a[g.bin[p]].add((i128)fw.W[i] * fw.W[g.nbr[p]]);
    }
  for (int b = 0; b < g.nb; ++b) {
    if (pairs) pairs[b] = c[b];
    if (wpairs) wpairs[b] = w ? a[b].to_double(2 * fw.S) : (double)c[b];
  }
  return 0;
}

// Sec. 3.3, Eq. (disc). rr == NULL selects the analytic periodic-box random
// pair count RR[b] = P * V_b / V_box with V_b = (4 pi / 3)(E_{b+1}^3 - E_b^3)
// and P = N(N-1)/2 (unweighted) or ((sum w)^2 - sum w^2)/2 (weighted).
// xi[b] = pairsum[b] / RR[b] - 1. zeta_disc over the 4-point orbits.
// Returns -1 when rr is NULL in an open box.
int or_disconnected(void* gp, const float* w, const double* rr, uint64_t* pairs, double* xi,
                    double* zeta_disc) {
  Graph& g = *(Graph*)gp;
  std::vector<uint64_t> pc(g.nb);
  std::vector<double> pw(g.nb);
  int st = or_pairs(gp, w, pc.data(), pw.data());
  if (st) return st;
  if (pairs) std::memcpy(pairs, pc.data(), sizeof(uint64_t) * g.nb);
  std::vector<double> RR(g.nb);
  if (rr) {
    for (int b = 0; b < g.nb; ++b) RR[b] = rr[b];
  } else {
    if (g.box_u <= 0) return -1;
    double P;
    if (w) {
      FixedWeights fw = make_fixed(w, g.n);
      Acc256 s1, s2;
      for (int64_t i = 0; i < g.n; ++i) {
        s1.add((i128)fw.W[i]);
        s2.add((i128)fw.W[i] * fw.W[i]);
      }
      const double S1 = s1.to_double(fw.S), S2 = s2.to_double(2 * fw.S);
      P = (S1 * S1 - S2) / 2.0;
    } else {
      P = (double)g.n * (double)(g.n - 1) / 2.0;
    }
    const i128 L = g.box_u;
    const double vbox = (double)(L * L * L);
    const double four_pi_3 = 4.0 * M_PI / 3.0;
    for (int b = 0; b < g.nb; ++b) {
      const i128 e1 = g.edges[b + 1], e0 = g.edges[b];
      const double dv = (double)(e1 * e1 * e1 - e0 * e0 * e0);
      const double vb = four_pi_3 * dv;
      RR[b] = P * vb / vbox;
    }
  }
  std::vector<double> x(g.nb);
  for (int b = 0; b < g.nb; ++b) {
    const double num = w ? pw[b] : (double)pc[b];
    x[b] = num / RR[b] - 1.0;
    if (xi) xi[b] = x[b];
  }
  if (zeta_disc) {
    Conf4* conf = conf4_cached(g.nb);
    for (size_t o = 0; o < conf->reps.size(); ++o) {
      const Tup6& r = conf->reps[o];
      // slots: 0=01 1=02 2=03 3=12 4=13 5=23
      volatile double t1 = x[r[0]] * x[r[5]];
      volatile double t2 = x[r[1]] * x[r[4]];
      volatile double t3 = x[r[2]] * x[r[3]];
      volatile double s = t1 + t2;
      zeta_disc[o] = s + t3;
    }
  }
  return 0;
}

// Sec. 3.3 (Eq. disc, Eq. conn) with the signed-weight estimator of Sec. 2.1:
// g_dr holds data and randoms together with data weights summing to +1 and
// random weights to -1; g_r holds the randoms alone with weights summing to
// +1. Then, per radial bin and per 4-point configuration,
//   xi        = (signed pair sum) / (random pair sum), no additive constant;
//   zeta_even = NNNN_even / RRRR, zeta_odd = NNNN_odd / RRRR;
//   zeta_disc = Eq. (disc) on xi; zeta_conn = zeta_even - zeta_disc
// (the disconnected part is parity-even and leaves the odd channel alone).
// Any output may be NULL. Returns 0, -2 when weights cannot be summed exactly.
int or_connected_4pcf(void* g_dr, const float* w_signed, void* g_r, const float* w_r, double* xi,
                      double* zeta_even, double* zeta_odd, double* zeta_disc, double* zeta_conn,
                      int nthreads) {
  Graph& gd = *(Graph*)g_dr;
  Graph& gr = *(Graph*)g_r;
  if (gd.nb != gr.nb) return -1;
  const int nb = gd.nb;
  Conf4* conf = conf4_cached(nb);
  const size_t nc = conf->reps.size();
  std::vector<uint64_t> pc(nb);
  std::vector<double> nn(nb), rr(nb);
  int st = or_pairs(g_dr, w_signed, pc.data(), nn.data());
  if (!st) st = or_pairs(g_r, w_r, pc.data(), rr.data());
  if (st) return st;
  std::vector<uint64_t> e(nc);
  std::vector<int64_t> o(nc);
  std::vector<double> ne(nc), no(nc), re(nc), ro(nc);
  st = or_count_4pcf(g_dr, w_signed, e.data(), o.data(), ne.data(), no.data(), nthreads);
  if (!st) st = or_count_4pcf(g_r, w_r, e.data(), o.data(), re.data(), ro.data(), nthreads);
  if (st) return st;
  std::vector<double> x(nb);
  for (int b = 0; b < nb; ++b) {
    x[b] = nn[b] / rr[b];
    if (xi) xi[b] = x[b];
  }
  for (size_t c = 0; c < nc; ++c) {
    const Tup6& r = conf->reps[c];
    volatile double t1 = x[r[0]] * x[r[5]];
    volatile double t2 = x[r[1]] * x[r[4]];
    volatile double t3 = x[r[2]] * x[r[3]];
    volatile double s12 = t1 + t2;
    const double disc = s12 + t3;
    const double ze = ne[c] / re[c];
    if (zeta_even) zeta_even[c] = ze;
    if (zeta_odd) zeta_odd[c] = no[c] / re[c];
    if (zeta_disc) zeta_disc[c] = disc;
    if (zeta_conn) {
      volatile double zc = ze - disc;
      zeta_conn[c] = zc;
    }
  }
  return 0;
}

}  // extern "C"
