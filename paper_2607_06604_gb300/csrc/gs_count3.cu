// Binned triangle counts (Sec. 2.2) with the hub-and-spoke intersection of
// sorted rows (Sec. 3.1), GB300 layout.
//
// For each hub i and spoke j in N+(i), the triangles (i, j, k) with k > j
// are k in N+(i) intersected with N+(j). The paper walks both sorted lists
// with two pointers per lane group; here a persistent CTA takes one hub at a
// time, stages N+(i) in shared memory with a bulk (TMA) copy, builds a
// shared-memory hash of it, and every warp streams the rows N+(j) of its
// spokes with 128-bit loads, four edge words per lane, probing the hash.
// A spoke row is read in ascending order and abandoned as soon as its ids
// pass the largest id of N+(i) (the merge-walk's exhaustion rule).
// Counts go to per-CTA shared-memory histograms over canonical
// configurations and are flushed with one 64-bit atomic per bin.
// Weighted sums use exact fixed point: per-triangle 128-bit products in
// shared 128-bit accumulators, flushed into 192-bit global accumulators.
#include <algorithm>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kSegCap = 2048;   // hub-row words staged per pass
constexpr int kHashCap = 8192;  // hash slots, >= 4 x staged words

struct Args {
  const int64_t* __restrict__ ptr;
  const int32_t* __restrict__ deg;
  const uint32_t* __restrict__ adj;  // row i at adj + (ptr[i] - adj_off)
  int64_t adj_off;
  int64_t hub_begin, hub_end;
  int nb, nconf;
  int seg_cap;  // hub-row words staged per pass (<= kSegCap, multiple of 4)
  unsigned long long* counts;  // [nconf]
  unsigned long long* wacc;    // [nconf][3] 192-bit
  const int64_t* __restrict__ W;
  unsigned long long* hub_counter;
  int* err;
};

template <bool WEIGHTED, bool SMEM_HIST>
__global__ void __launch_bounds__(kThreads) k_count3(Args a) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t* stage = reinterpret_cast<uint32_t*>(smem);
  uint32_t* table = stage + kSegCap;
  unsigned* hist = table + kHashCap;
  unsigned long long* whist =
      reinterpret_cast<unsigned long long*>(hist + ((a.nconf + 1) & ~1));
  __shared__ uint64_t bar;
  __shared__ int64_t s_hub;
  __shared__ unsigned long long s_pending;
  __shared__ int s_flush;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (SMEM_HIST) {
    for (int k = tid; k < a.nconf; k += kThreads) hist[k] = 0;
    if (WEIGHTED)
      for (int k = tid; k < 2 * a.nconf; k += kThreads) whist[k] = 0;
  }
  if (tid == 0) {
    mbar_init(&bar, 1);
    s_pending = 0;
  }
  __syncthreads();
  uint32_t phase = 0;

  auto flush = [&]() {
    if (!SMEM_HIST) return;
    for (int k = tid; k < a.nconf; k += kThreads) {
      const unsigned c = hist[k];
      if (c) {
        atomicAdd(a.counts + k, (unsigned long long)c);
        hist[k] = 0;
      }
    }
  };

  for (;;) {
    if (tid == 0) {
      s_hub = a.hub_begin + (int64_t)atomicAdd(a.hub_counter, 1ull);
      s_flush = 0;
      if (s_hub < a.hub_end) {
        const unsigned long long d = (unsigned long long)a.deg[s_hub];
        const unsigned long long need = d * (d - (d > 0)) / 2;  // triangles at i <= C(d,2)
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
    if (i >= a.hub_end) break;
    if (s_flush) {
      flush();
      __syncthreads();
    }
    const int d = a.deg[i];
    if (d < 2) {
      __syncthreads();
      continue;
    }
    const uint32_t* row = a.adj + (a.ptr[i] - a.adj_off);
    const int64_t Wi = WEIGHTED ? a.W[i] : 0;
    const int seg_cap = a.seg_cap;
    for (int s0 = 0; s0 < d; s0 += seg_cap) {
      const int sn = min(seg_cap, d - s0);
      const int sn4 = (int)pad_row(sn);
      if (tid == 0) bulk_load(stage, row + s0, (uint32_t)sn4 * 4u, &bar);
      int tbits = 7;
      while ((1 << tbits) < 4 * sn && tbits < 13) ++tbits;
      const int T = 1 << tbits;
      const int shift = 32 - tbits;
      for (int k = tid; k < T; k += kThreads) table[k] = kSentinel;
      const bool ok = mbar_wait(&bar, phase, kWaitLimit);
      phase ^= 1u;
      if (__syncthreads_or(!ok)) {
        if (tid == 0) atomicOr(a.err, kErrTimeout);
        return;
      }
      for (int k = tid; k < sn; k += kThreads) {
        const uint32_t w = stage[k];
        uint32_t h = (edge_id(w) * kHashMul) >> shift;
        while (atomicCAS(table + h, kSentinel, w) != kSentinel) h = (h + 1) & (T - 1);
      }
      __syncthreads();
      const uint32_t seg_lo = edge_id(stage[0]);
      const uint32_t seg_hi = edge_id(stage[sn - 1]);
      for (int sp = warp; sp < d; sp += kWarps) {
        const uint32_t wij = (d <= seg_cap) ? stage[sp] : row[sp];
        const uint32_t j = edge_id(wij);
        if (j >= seg_hi) break;  // every k > j; none left in this segment
        const int bij = (int)edge_bin(wij);
        const int64_t Wij = WEIGHTED ? Wi * a.W[j] : 0;
        const uint32_t* rj = a.adj + (a.ptr[j] - a.adj_off);
        const int dj4 = (int)pad_row(a.deg[j]);
        int start = 0;
        if (s0 > 0) {  // skip to the first id >= seg_lo (rows are sorted)
          int lo = 0, hi = a.deg[j];
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
            if (key > seg_hi) continue;
            uint32_t h = (key * kHashMul) >> shift;
            for (;;) {
              const uint32_t e = table[h];
              if (e == kSentinel) break;
              if (edge_id(e) == key) {
                const int c = conf3_rank(bij, (int)edge_bin(e), (int)edge_bin(vv[q]), a.nb);
                if (SMEM_HIST) atomicAdd(hist + c, 1u);
                else atomicAdd(a.counts + c, 1ull);
                if (WEIGHTED) {
                  long long lo, hi;
                  mul_i128(Wij, a.W[key], &lo, &hi);
                  if (SMEM_HIST) atomic_add_i128(whist + 2 * c, lo, hi);
                  else atomic_add_i192(a.wacc + 3 * c, (unsigned long long)lo, (unsigned long long)hi);
                }
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
    }
  }
  __syncthreads();
  flush();
  if (SMEM_HIST && WEIGHTED) {
    for (int k = tid; k < a.nconf; k += kThreads) {
      const unsigned long long lo = whist[2 * k], hi = whist[2 * k + 1];
      if (lo | hi) atomic_add_i192(a.wacc + 3 * k, lo, hi);
    }
  }
}

}  // namespace

// 192-bit two's-complement integer times 2^-scale, to double (the top 64
// significant bits, then one rounding).
__global__ void k_i192_to_double(const unsigned long long* acc, int64_t n, int scale,
                                 double* out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long m[3] = {acc[3 * k], acc[3 * k + 1], acc[3 * k + 2]};
    const bool neg = (m[2] >> 63) != 0;
    if (neg) {
      unsigned long long c = 1;
      for (int q = 0; q < 3; ++q) {
        const unsigned long long x = ~m[q];
        const unsigned long long s = x + c;
        c = (s < x) ? 1ull : 0ull;
        m[q] = s;
      }
    }
    int top = -1;
    for (int q = 2; q >= 0; --q)
      if (m[q]) {
        top = q;
        break;
      }
    double v = 0.0;
    if (top >= 0) {
      const int msb = top * 64 + 63 - __clzll((long long)m[top]);
      int shift = msb - 63;
      unsigned long long mant;
      if (shift <= 0) {
        mant = m[0];
        shift = 0;
      } else {
        const int ws = shift / 64, bs = shift % 64;
        const unsigned long long lo = m[ws], hi = (ws + 1 < 3) ? m[ws + 1] : 0ull;
        mant = bs ? ((lo >> bs) | (hi << (64 - bs))) : lo;
      }
      v = ldexp((double)mant, shift - scale);
    }
    out[k] = neg ? -v : v;
  }
}

__global__ void k_u64_to_double(const unsigned long long* c, int64_t n, double* out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    out[k] = (double)c[k];
}

int count3_device(const Graph& g, const FixedW* fw, uint64_t* d_counts, double* d_wsum,
                  const Opts& o, Scratch& sc) {
  cudaStream_t s = o.stream;
  const int nconf = (int)num_conf3(g.nb);
  Args a;
  a.ptr = g.d_ptr;
  a.deg = g.d_deg;
  a.adj = nullptr;
  a.adj_off = 0;
  a.nb = g.nb;
  a.nconf = nconf;
  // variant 1 stages 64-word segments: exercises the long-row path on any input
  a.seg_cap = (o.variant & 1) ? 64 : kSegCap;
  a.counts = reinterpret_cast<unsigned long long*>(d_counts);
  a.W = fw ? fw->d_W : nullptr;
  const bool weighted = fw && d_wsum;
  a.wacc = weighted ? sc.alloc<unsigned long long>(3 * (size_t)nconf) : nullptr;
  a.hub_counter = sc.alloc<unsigned long long>(1);
  a.err = sc.alloc<int>(1);
  if (!a.hub_counter || !a.err || (weighted && !a.wacc)) return GS_ENOMEM;
  cudaMemsetAsync(d_counts, 0, sizeof(uint64_t) * nconf, s);
  if (weighted) cudaMemsetAsync(a.wacc, 0, sizeof(unsigned long long) * 3 * nconf, s);
  cudaMemsetAsync(a.err, 0, sizeof(int), s);
  if (g.n == 0) {
    if (d_wsum) cudaMemsetAsync(d_wsum, 0, sizeof(double) * nconf, s);
    return cuda_status(cudaGetLastError());
  }

  const size_t base = (size_t)(kSegCap + kHashCap) * 4;
  const size_t hist_bytes = (size_t)((nconf + 1) & ~1) * 4 + (weighted ? (size_t)nconf * 16 : 0);
  const bool smem_hist = hist_bytes <= 96 * 1024;
  const size_t smem = base + (smem_hist ? hist_bytes : 0);
  void (*kern)(Args);
  if (weighted) kern = smem_hist ? k_count3<true, true> : k_count3<true, false>;
  else kern = smem_hist ? k_count3<false, true> : k_count3<false, false>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0, sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
  const int grid = std::max(1, per_sm) * sms;
  KernelTimer timer(o.kernel_ms);
  timer.start(s);
  int st = for_each_window(g, o, sc, [&](const uint32_t* adj, int64_t off, int64_t h0,
                                         int64_t h1) -> int {
    a.adj = adj;
    a.adj_off = off;
    a.hub_begin = h0;
    a.hub_end = h1;
    cudaMemsetAsync(a.hub_counter, 0, sizeof(unsigned long long), s);
    { kern<<<grid, kThreads, smem, s>>>(a); note_launch(); }
    return cuda_status(cudaGetLastError());
  });
  timer.stop(s);
  if (st) return st;
  cudaError_t e;
  if (d_wsum) {
    if (weighted)
      { k_i192_to_double<<<(nconf + 255) / 256, 256, 0, s>>>(a.wacc, nconf, 3 * fw->scale, d_wsum); note_launch(); }
    else
      { k_u64_to_double<<<(nconf + 255) / 256, 256, 0, s>>>(a.counts, nconf, d_wsum); note_launch(); }
  }
  int herr = 0;
  cudaMemcpyAsync(&herr, a.err, sizeof(int), cudaMemcpyDeviceToHost, s);
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e);
  timer.publish();
  return herr ? GS_ETIMEOUT : GS_OK;
}

}  // namespace gs
