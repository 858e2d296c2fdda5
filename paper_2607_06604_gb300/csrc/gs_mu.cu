// Anisotropic 3pCF: triangle counts binned by configuration and by mu, the
// orientation of the triangle's plane against the line of sight. The paper
// names mu binning for redshift-space distortions (conclusions) without
// defining it; the reading built here: the line of sight is the z axis (a
// distant observer, as in a simulation box), a triangle's mu is |n_z| / |n|
// for the normal n = d_ij x d_ik of its plane (no relabelling of the
// vertices changes it), its bin the largest m < nmu with m / nmu <= mu, and
// collinear triangles (n = 0) go to the extra bin nmu.
//
// Kernel: the pair geometry of the triangle kernel. A persistent CTA takes
// one hub i at a time, stages the hub-relative displacement of every
// neighbour (and its hub-edge bin), and tests every pair (j, k) of N+(i):
// an edge exactly when E_0^2 <= |D_k - D_j|^2 < E_nb^2. For each triangle
// the normal D_j x D_k is formed in 64-bit integers (E_nb < 2^27) and the
// mu bin decided exactly by comparing m^2 |n|^2 with nmu^2 n_z^2 in 128-bit
// integers, starting from a floating-point guess that is corrected by
// those comparisons. Counts go to per-CTA shared histograms of
// nconf (nmu + 1) cells when they fit (global 64-bit atomics otherwise);
// weighted sums of W_i W_j W_k go straight to 192-bit global sums.
#include <algorithm>
#include <cmath>

#include "gs_internal.cuh"

namespace gs {

__global__ void k_i192_to_double(const unsigned long long* acc, int64_t n, int scale, double* out);
__global__ void k_u64_to_double(const unsigned long long* c, int64_t n, double* out);

namespace {

constexpr int kMThreads = 512;
constexpr int kMCap = 2048;  // neighbours staged in shared memory
constexpr int kMBucketMax = 2048;

struct MArgs {
  const int64_t* __restrict__ ptr;
  const int32_t* __restrict__ deg;
  const uint32_t* __restrict__ adj;  // row i at row_at(adj, ptr, i, adj_off, split, adj_off2)
  int64_t adj_off, split, adj_off2;
  int64_t hub_begin, hub_end;
  const int4* __restrict__ xyzp;
  int64_t box;
  const int64_t* __restrict__ W;  // fixed-point weights, or nullptr
  const int64_t* __restrict__ e2g;
  int nb, nconf, nmu;
  int cap;        // neighbours staged in shared memory
  int bk_shift, bk_n;  // squared-distance buckets (bk_n = 0: binary search)
  int smem_hist;  // 1: shared histogram of nconf (nmu + 1) counts
  int use_lut;    // 1: configuration ranks from a shared table over (b_ij, b_ik, b_jk)
  unsigned long long* counts;  // [nconf][nmu + 1]
  unsigned long long* wacc;    // [nconf][nmu + 1][3] 192-bit sums, or nullptr
  unsigned long long* hub_counter;
  unsigned char* gscratch;  // rows longer than cap: per-CTA staging
  size_t gstride;
};

// Unsigned 128-bit values as (hi, lo) 64-bit words, with the few
// operations the mu comparisons need.
struct U128 {
  unsigned long long hi, lo;
};
__device__ inline U128 square(long long v) {
  const unsigned long long a = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
  return U128{__umul64hi(a, a), a * a};
}
__device__ inline U128 add(const U128& x, const U128& y) {
  const unsigned long long lo = x.lo + y.lo;
  return U128{x.hi + y.hi + (lo < x.lo ? 1ull : 0ull), lo};
}
__device__ inline U128 times(const U128& x, unsigned k) {  // no overflow for the values met here
  return U128{x.hi * k + __umul64hi(x.lo, (unsigned long long)k), x.lo * k};
}
__device__ inline bool le(const U128& a, const U128& b) {
  return a.hi < b.hi || (a.hi == b.hi && a.lo <= b.lo);
}

// mu bin of a normal (nx, ny, nz), components below 2^39 in magnitude (the
// graph keeps E_nb below 2^19): the largest m in [0, nmu) with
// m^2 |n|^2 <= nmu^2 nz^2 (at most 2^124), nmu
// for n = 0. t = nmu |nz| / |n| in single precision carries a relative
// error below 12 2^-24 (the conversions, three products, two sums, the
// reciprocal square root's 2 ulp and two more products), so below 2^-14
// absolutely for nmu <= 64: when t lies at least 2^-10 from every integer,
// floor(t) is the bin. Otherwise the exact comparisons decide.
__device__ inline int mu_bin(long long nx, long long ny, long long nz, int nmu) {
  if ((nx | ny | nz) == 0) return nmu;
  const float fx = i40_to_float(nx), fy = i40_to_float(ny), fz = i40_to_float(nz);
  const float t = (float)nmu * fabsf(fz) * rsqrtf(fx * fx + fy * fy + fz * fz);
  const float r = rintf(t);
  if (fabsf(t - r) >= 0.0009765625f) {
    const int m = (int)t;
    return m > nmu - 1 ? nmu - 1 : m;
  }
  const U128 z2 = square(nz);
  const U128 n2 = add(add(square(nx), square(ny)), z2);
  const U128 rhs = times(z2, (unsigned)(nmu * nmu));
  int m = (int)r;
  m = m < 0 ? 0 : (m > nmu - 1 ? nmu - 1 : m);
  while (m > 0 && !le(times(n2, (unsigned)(m * m)), rhs)) --m;
  while (m + 1 < nmu && le(times(n2, (unsigned)((m + 1) * (m + 1))), rhs)) ++m;
  return m;
}

// SMALL: E_nb <= 2^16, so a pair with any |component| >= 2^16 is no edge
// and otherwise each squared component fits 32 bits.
template <bool WEIGHTED, bool SMALL>
__global__ void __launch_bounds__(kMThreads, 2) k_count3mu(MArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  int4* s_stage = reinterpret_cast<int4*>(smem);
  int* s_w = reinterpret_cast<int*>(s_stage + a.cap);
  unsigned* hist = reinterpret_cast<unsigned*>(s_w + (WEIGHTED ? a.cap : 0));
  uint16_t* s_lut = reinterpret_cast<uint16_t*>(hist + (a.smem_hist ? a.nconf * (a.nmu + 1) : 0));
  __shared__ int64_t s_e2[kMaxBins + 1];
  __shared__ uint8_t s_bk[kMBucketMax];
  __shared__ int64_t s_hub;
  __shared__ unsigned long long s_pending;
  __shared__ int s_flush, s_next;
  const int tid = threadIdx.x, lane = tid & 31;
  const int nb = a.nb, nm1 = a.nmu + 1;
  const int ncell = a.nconf * nm1;
  for (int b = tid; b <= nb; b += kMThreads) s_e2[b] = a.e2g[b];
  // bucket k covers squared distances [k 2^shift, (k + 1) 2^shift) and holds
  // at most one bin edge; it stores the bin of its start
  for (int k = tid; k < a.bk_n; k += kMThreads) {
    const int64_t x = (int64_t)k << a.bk_shift;
    int b = 0;
    while (b + 1 < nb && a.e2g[b + 1] <= x) ++b;
    s_bk[k] = (uint8_t)b;
  }
  if (a.smem_hist)
    for (int k = tid; k < ncell; k += kMThreads) hist[k] = 0u;
  if (a.use_lut)
    for (int k = tid; k < nb * nb * nb; k += kMThreads)
      s_lut[k] = (uint16_t)conf3_rank(k / (nb * nb), (k / nb) % nb, k % nb, nb);
  if (tid == 0) s_pending = 0;
  __syncthreads();
  const int64_t e2lo = s_e2[0], e2hi = s_e2[nb];

  auto flush = [&]() {
    if (!a.smem_hist) return;
    for (int k = tid; k < ncell; k += kMThreads) {
      const unsigned v = hist[k];
      if (v) {
        atomicAdd(a.counts + k, (unsigned long long)v);
        hist[k] = 0u;
      }
    }
  };

  for (;;) {
    if (tid == 0) {
      const int64_t i = a.hub_begin + (int64_t)atomicAdd(a.hub_counter, 1ull);
      s_hub = i < a.hub_end ? i : -1;
      s_flush = 0;
      s_next = 0;
      if (i < a.hub_end) {
        const unsigned long long d = (unsigned long long)a.deg[i];
        const unsigned long long need = d * (d - (d > 0)) / 2;  // triangles at i <= C(d, 2)
        if (s_pending + need > 0xFFFFFFFFull) {
          s_flush = 1;
          s_pending = need;
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
    const int d = a.deg[i];
    if (d < 2) {
      __syncthreads();
      continue;
    }
    const uint32_t* row = row_at(a.adj, a.ptr, i, a.adj_off, a.split, a.adj_off2);
    const int4 P = a.xyzp[i];
    const bool big = d > a.cap;
    int4* S = big ? reinterpret_cast<int4*>(a.gscratch + (size_t)blockIdx.x * a.gstride) : s_stage;
    int* SW = big ? reinterpret_cast<int*>(S + d) : s_w;
    for (int t = tid; t < d; t += kMThreads) {
      const uint32_t w = row[t];
      const uint32_t k = edge_id(w);
      const int4 Q = a.xyzp[k];
      auto mi = [&](int64_t x) {
        if (a.box) {
          if (2 * x >= a.box) x -= a.box;
          else if (2 * x < -a.box) x += a.box;
        }
        return (int)x;
      };
      S[t] = make_int4(mi((int64_t)Q.x - P.x), mi((int64_t)Q.y - P.y), mi((int64_t)Q.z - P.z),
                       (int)edge_bin(w));
      if (WEIGHTED) SW[t] = (int)a.W[k];
    }
    __syncthreads();
    const int64_t Wi = WEIGHTED ? a.W[i] : 0;
    for (;;) {
      int ra = 0;
      if (lane == 0) ra = atomicAdd(&s_next, 1);
      ra = __shfl_sync(0xffffffffu, ra, 0);
      if (ra >= d - 1) break;
      const int4 Da = S[ra];
      const int64_t Wia = WEIGHTED ? Wi * SW[ra] : 0;
      const int abase = Da.w * nb * nb;
      for (int rb = ra + 1 + lane; rb < d; rb += 32) {
        const int4 Db = S[rb];
        int64_t D2;
        if constexpr (SMALL) {
          const unsigned ax = (unsigned)abs(Db.x - Da.x), ay = (unsigned)abs(Db.y - Da.y),
                         az = (unsigned)abs(Db.z - Da.z);
          if (max(ax, max(ay, az)) >= 65536u) continue;
          D2 = (int64_t)((unsigned long long)(ax * ax) + (ay * ay) + (az * az));
        } else {
          const int64_t x = (int64_t)Db.x - Da.x, y = (int64_t)Db.y - Da.y,
                        z = (int64_t)Db.z - Da.z;
          D2 = x * x + y * y + z * z;
        }
        if (D2 < e2lo || D2 >= e2hi) continue;
        int lo;
        if (a.bk_n) {
          lo = s_bk[D2 >> a.bk_shift];
          lo += D2 >= s_e2[lo + 1] ? 1 : 0;
        } else {
          lo = 0;
          int hi = nb;
          while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (s_e2[mid] <= D2) lo = mid;
            else hi = mid;
          }
        }
        const int cf = a.use_lut ? (int)s_lut[abase + Db.w * nb + lo] : conf3_rank(Da.w, Db.w, lo, nb);
        const long long nx = (long long)Da.y * Db.z - (long long)Da.z * Db.y;
        const long long ny = (long long)Da.z * Db.x - (long long)Da.x * Db.z;
        const long long nz = (long long)Da.x * Db.y - (long long)Da.y * Db.x;
        const int cell = cf * nm1 + mu_bin(nx, ny, nz, a.nmu);
        if (a.smem_hist) atomicAdd(hist + cell, 1u);
        else atomicAdd(a.counts + cell, 1ull);
        if (WEIGHTED) {
          long long plo, phi;
          mul_i128(Wia, (long long)SW[rb], &plo, &phi);
          atomic_add_i192(a.wacc + 3 * cell, (unsigned long long)plo, (unsigned long long)phi);
        }
      }
    }
    __syncthreads();
  }
  __syncthreads();
  flush();
}

}  // namespace

int count3mu_device(const Graph& g, const FixedW* fw, int nmu, uint64_t* d_counts,
                    double* d_wsum, const Opts& o, Scratch& sc) {
  cudaStream_t s = o.stream;
  if (nmu < 1 || nmu > 64) return GS_EINVAL;
  // the normal's components stay below 2^55 and the exact mu comparisons
  // below 2^124 when E_nb < 2^27 (graphs are built with E_nb < 2^19)
  if (g.edges[g.nb] >= (int64_t(1) << 27)) return GS_ERANGE;
  const int nconf = (int)num_conf3(g.nb);
  const int64_t ncell = (int64_t)nconf * (nmu + 1);
  const bool weighted = fw != nullptr;
  MArgs a;
  a.ptr = g.d_ptr;
  a.deg = g.d_deg;
  a.adj = nullptr;
  a.adj_off = 0;
  a.split = g.n;
  a.adj_off2 = 0;
  a.xyzp = g.d_xyzp;
  a.box = g.box_u;
  a.W = weighted ? fw->d_W : nullptr;
  a.e2g = g.d_edges2;
  a.nb = g.nb;
  a.nconf = nconf;
  a.nmu = nmu;
  a.counts = reinterpret_cast<unsigned long long*>(d_counts);
  a.wacc = weighted ? sc.alloc<unsigned long long>(3 * (size_t)ncell) : nullptr;
  a.hub_counter = sc.alloc<unsigned long long>(1);
  if (!a.hub_counter || (weighted && !a.wacc)) return GS_ENOMEM;
  cudaMemsetAsync(d_counts, 0, sizeof(uint64_t) * ncell, s);
  if (weighted) cudaMemsetAsync(a.wacc, 0, sizeof(unsigned long long) * 3 * ncell, s);

  int dev = 0, sms = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  // staging capacity: the longest row (rows above kMCap are staged in
  // global memory)
  a.cap = std::min(kMCap, std::max(32, (g.max_deg + 31) & ~31));
  // squared-distance buckets no wider than the narrowest bin
  a.bk_shift = 0;
  a.bk_n = 0;
  {
    int64_t gap = INT64_MAX;
    for (int b = 0; b < g.nb; ++b)
      gap = std::min(gap, g.edges[b + 1] * g.edges[b + 1] - g.edges[b] * g.edges[b]);
    int sh = 0;
    while (sh < 62 && (int64_t(1) << (sh + 1)) <= gap) ++sh;
    const int64_t top = g.edges[g.nb] * g.edges[g.nb];
    const int64_t nbk = ((top - 1) >> sh) + 1;
    if (gap >= 1 && nbk <= kMBucketMax) {
      a.bk_shift = sh;
      a.bk_n = (int)nbk;
    }
  }
  const size_t stage = (size_t)a.cap * (weighted ? 20 : 16);
  const size_t hist = (size_t)ncell * 4;
  const size_t lut = ((size_t)g.nb * g.nb * g.nb * 2 + 15) & ~(size_t)15;
  const size_t avail = (size_t)optin - 8 * (kMaxBins + 1) - kMBucketMax - 256;
  a.smem_hist = stage + hist <= avail ? 1 : 0;
  // the table too when two CTAs per SM still fit
  int per_sm_bytes = 0;
  cudaDeviceGetAttribute(&per_sm_bytes, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  const size_t two = (size_t)per_sm_bytes / 2 - 1024 - 8 * (kMaxBins + 1) - kMBucketMax - 256;
  const size_t base = stage + (a.smem_hist ? hist : 0);
  a.use_lut = (a.smem_hist && base + lut <= two) ? 1 : 0;
  const size_t smem = base + (a.use_lut ? lut : 0);
  const bool small = g.edges[g.nb] <= 65536;
  void (*kern)(MArgs) = weighted ? (small ? k_count3mu<true, true> : k_count3mu<true, false>)
                                 : (small ? k_count3mu<false, true> : k_count3mu<false, false>);
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kMThreads, smem);
  const int grid = std::max(1, per_sm) * sms;
  a.gscratch = nullptr;
  a.gstride = 0;
  if (g.max_deg > a.cap) {
    a.gstride = ((size_t)g.max_deg * 20 + 255) & ~(size_t)255;
    a.gscratch = sc.alloc<unsigned char>(a.gstride * grid);
    if (!a.gscratch) return GS_ENOMEM;
  }
  KernelTimer timer(o.kernel_ms);
  timer.start(s);
  int st = GS_OK;
  if (g.n > 0)
    st = for_each_window(g, o, sc, [&](const WinView& v) -> int {
      a.adj = v.adj;
      a.adj_off = v.off1;
      a.split = v.split;
      a.adj_off2 = v.off2;
      a.hub_begin = v.h0;
      a.hub_end = v.h1;
      cudaMemsetAsync(a.hub_counter, 0, sizeof(unsigned long long), s);
      { kern<<<grid, kMThreads, smem, s>>>(a); note_launch(); }
      return cuda_status(cudaGetLastError());
    });
  if (st) return st;
  timer.stop(s);
  if (d_wsum) {
    const int blocks = (int)std::min<int64_t>((ncell + 255) / 256, 4096);
    if (weighted)
      { k_i192_to_double<<<blocks, 256, 0, s>>>(a.wacc, ncell, 3 * fw->scale, d_wsum); note_launch(); }
    else
      { k_u64_to_double<<<blocks, 256, 0, s>>>(a.counts, ncell, d_wsum); note_launch(); }
  }
  const cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e);
  timer.publish();
  return cuda_status(cudaGetLastError());
}

}  // namespace gs
