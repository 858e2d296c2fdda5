// Equilateral 3pCF: triangles whose three sides fall in the same radial bin
// (the configurations (b, b, b) of the full 3pCF), from the oriented graph
// of Sec. 2.1 with the enumeration of Sec. 2.2.
//
// Only same-bin edges can close such a triangle, so a spoke j of bin b in
// N+(i) keeps the words of N+(j) whose bin is b (a register test on the low
// byte) and looks each kept id up in N+(i) by binary search. The lookup
// compares whole edge words, so it checks id and bin together. About one
// word in nb reaches the lookup, so the kernel spends its time streaming the
// spoke rows, with 128-bit loads, and abandons a spoke row once its ids pass
// the largest id of N+(i) (the merge-walk's exhaustion rule of Sec. 3.1).
// Hub i's row is staged in shared memory when it fits. Counts
// and weight sums build up in registers for each spoke and reach shared
// memory once per spoke.
#include <algorithm>

#include "gs_internal.cuh"

namespace gs {

__global__ void k_i192_to_double(const unsigned long long* acc, int64_t n, int scale, double* out);

namespace {

constexpr int kEqThreads = 256;
constexpr int kEqWarps = kEqThreads / 32;
constexpr int kEqStage = 4096;  // staged words of the hub row (16 KB)
// flush the block's 128-bit weight sums after this many triangles: each
// product W_i W_j W_k is below 2^90, so 2^36 of them stay below 2^127
constexpr unsigned long long kEqFlushTri = 1ull << 36;

template <bool WEIGHTED>
__global__ void __launch_bounds__(kEqThreads) k_equi3(const int64_t* __restrict__ ptr,
                                                      const int32_t* __restrict__ deg, WinView v,
                                                      const int64_t* __restrict__ W, int nb,
                                                      unsigned long long* hub_counter,
                                                      unsigned long long* counts,
                                                      unsigned long long* wacc) {
  __shared__ __align__(16) uint32_t srow[kEqStage];
  __shared__ unsigned long long s_cnt[kMaxBins + 1];
  __shared__ unsigned long long s_w[2 * (kMaxBins + 1)];
  __shared__ unsigned long long s_tri;
  __shared__ int64_t s_hub;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int b = tid; b < nb; b += kEqThreads) {
    s_cnt[b] = 0;
    s_w[2 * b] = s_w[2 * b + 1] = 0;
  }
  if (tid == 0) s_tri = 0;
  auto flush = [&]() {
    for (int b = tid; b < nb; b += kEqThreads) {
      if (s_cnt[b]) atomicAdd(counts + b, s_cnt[b]);
      s_cnt[b] = 0;
      if (WEIGHTED && (s_w[2 * b] | s_w[2 * b + 1])) atomic_add_i192(wacc + 3 * b, s_w[2 * b], s_w[2 * b + 1]);
      s_w[2 * b] = s_w[2 * b + 1] = 0;
    }
  };
  for (;;) {
    __syncthreads();  // the previous hub's staged row is no longer read
    if (tid == 0) {
      s_hub = v.h0 + (int64_t)atomicAdd(hub_counter, 1ull);
      if (WEIGHTED && s_tri >= kEqFlushTri) s_tri = ~0ull;  // ask for a flush below
    }
    __syncthreads();
    if (WEIGHTED && s_tri == ~0ull) {
      flush();
      __syncthreads();
      if (tid == 0) s_tri = 0;
      __syncthreads();
    }
    const int64_t i = s_hub;
    if (i >= v.h1) break;
    const int d = deg[i];
    if (d < 2) continue;
    const uint32_t* gi = row_at(v.adj, ptr, i, v.off1, v.split, v.off2);
    const bool staged = d <= kEqStage;
    if (staged) {
      uint4* dst = reinterpret_cast<uint4*>(srow);
      for (int k = tid; k < (int)(pad_row(d) / 4); k += kEqThreads) dst[k] = ldg_nc_v4(gi + 4 * k);
      __syncthreads();
    }
    const uint32_t* ri = staged ? srow : gi;
    const int64_t Wi = WEIGHTED ? W[i] : 0;
    const uint32_t hub_hi = edge_id(ri[d - 1]);
    unsigned long long tri_warp = 0;
    const uint4 none = make_uint4(kSentinel, kSentinel, kSentinel, kSentinel);
    // The warp takes spokes q = warp, warp + kEqWarps, ...; the next spoke's
    // row pointer, length and first chunk are loaded while the current one
    // is walked, and so is the next chunk of the current row.
    int q = warp;
    uint32_t wj = 0;
    const uint32_t* rj = nullptr;
    int dj4 = 0;
    uint4 v0 = none;
    if (q < d - 1) {
      wj = ri[q];
      rj = row_at(v.adj, ptr, edge_id(wj), v.off1, v.split, v.off2);
      dj4 = (int)pad_row(deg[edge_id(wj)]);
      v0 = (lane * 4 < dj4) ? ldg_nc_v4(rj + lane * 4) : none;
    }
    while (q < d - 1) {
      const int qn = q + kEqWarps;
      uint32_t wjn = 0;
      const uint32_t* rjn = nullptr;
      int dj4n = 0;
      uint4 vn0 = none;
      if (qn < d - 1) {
        wjn = ri[qn];
        rjn = row_at(v.adj, ptr, edge_id(wjn), v.off1, v.split, v.off2);
        dj4n = (int)pad_row(deg[edge_id(wjn)]);
        vn0 = (lane * 4 < dj4n) ? ldg_nc_v4(rjn + lane * 4) : none;
      }
      const uint32_t b = edge_bin(wj);
      const int64_t j = edge_id(wj);
      int cnt = 0;
      int64_t sw = 0;
      // N+(j) in 128-word chunks (four edge words per lane, padded rows),
      // abandoned once its ids pass the largest id of N+(i)
      uint4 v4 = v0;
      for (int t0 = 0;; t0 += 128) {
        const uint32_t last = __shfl_sync(0xffffffffu, v4.w, 31);
        const bool more = edge_id(last) <= hub_hi && t0 + 128 < dj4;
        uint4 vnext = none;
        if (more) {
          const int t = t0 + 128 + lane * 4;
          vnext = (t < dj4) ? ldg_nc_v4(rj + t) : none;
        }
        const uint32_t vv[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) {
          const uint32_t wk = vv[qq];
          const uint32_t key = edge_id(wk);
          if (edge_bin(wk) != b || key > hub_hi) continue;
          // N+(i) holds ids above j only after position q
          int lo = q + 1, hi = d;
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (edge_id(ri[mid]) < key) lo = mid + 1;
            else hi = mid;
          }
          if (lo < d && ri[lo] == wk) {
            ++cnt;
            if (WEIGHTED) sw += W[key];
          }
        }
        if (!more) break;
        v4 = vnext;
      }
      for (int o = 16; o; o >>= 1) {
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        if (WEIGHTED) sw += __shfl_xor_sync(0xffffffffu, sw, o);
      }
      if (lane == 0 && cnt) {
        atomicAdd(s_cnt + b, (unsigned long long)cnt);
        tri_warp += (unsigned long long)cnt;
        if (WEIGHTED) {
          long long plo, phi;
          mul_i128(Wi * W[j], sw, &plo, &phi);
          atomic_add_i128(s_w + 2 * b, plo, phi);
        }
      }
      q = qn;
      wj = wjn;
      rj = rjn;
      dj4 = dj4n;
      v0 = vn0;
    }
    if (WEIGHTED && lane == 0 && tri_warp) atomicAdd(&s_tri, tri_warp);
  }
  __syncthreads();
  flush();
}

}  // namespace

int equi3_device(const Graph& g, const FixedW* fw, uint64_t* d_counts, double* d_wsum,
                 const Opts& o, Scratch& sc) {
  cudaStream_t s = o.stream;
  const int nb = g.nb;
  unsigned long long* counts = reinterpret_cast<unsigned long long*>(d_counts);
  unsigned long long* wacc = fw ? sc.alloc<unsigned long long>(3 * (size_t)nb) : nullptr;
  unsigned long long* hub_counter = sc.alloc<unsigned long long>(1);
  if (!hub_counter || (fw && !wacc)) return GS_ENOMEM;
  cudaMemsetAsync(counts, 0, sizeof(uint64_t) * nb, s);
  if (wacc) cudaMemsetAsync(wacc, 0, sizeof(unsigned long long) * 3 * nb, s);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  KernelTimer timer(o.kernel_ms);
  timer.start(s);
  int st = GS_OK;
  if (g.n)
    st = for_each_window(g, o, sc, [&](const WinView& v) -> int {
      cudaMemsetAsync(hub_counter, 0, sizeof(unsigned long long), s);
      if (fw)
        { k_equi3<true><<<sms * 4, kEqThreads, 0, s>>>(g.d_ptr, g.d_deg, v, fw->d_W, nb, hub_counter,
                                                      counts, wacc); note_launch(); }
      else
        { k_equi3<false><<<sms * 4, kEqThreads, 0, s>>>(g.d_ptr, g.d_deg, v, nullptr, nb, hub_counter,
                                                       counts, nullptr); note_launch(); }
      return cuda_status(cudaGetLastError());
    });
  timer.stop(s);
  if (st) return st;
  if (fw && d_wsum)
    { k_i192_to_double<<<(nb + 255) / 256, 256, 0, s>>>(wacc, nb, 3 * fw->scale, d_wsum); note_launch(); }
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e);
  timer.publish();
  return cuda_status(cudaGetLastError());
}

}  // namespace gs
