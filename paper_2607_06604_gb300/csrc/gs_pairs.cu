// Internal 2pCF and the disconnected 4pCF term (Sec. 3.3, Eq. disc).
//
// The unweighted pair histogram is one streaming pass over the packed edge
// words (the bin is the low byte of every word; padding words carry bin
// 0xFF and are skipped), 128-bit loads, per-CTA shared-memory counters.
// The weighted pass walks rows (warp per hub) to pair w_i with w_j, in
// exact fixed point. A single small kernel then forms RR, xi and
// zeta_disc in FP64 with explicitly rounded operations (no contraction),
// in the order the equation is written. The signed-weight estimator
// (connected 4pCF) reuses the weighted sweep and the 4pCF kernel.
#include <algorithm>

#include "gs_internal.cuh"

namespace gs {

__global__ void k_i192_to_double(const unsigned long long* acc, int64_t n, int scale, double* out);

namespace {

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_pairs_count(const uint4* __restrict__ adj4,
                                                          int64_t n4, int nb,
                                                          unsigned long long* pairs) {
  __shared__ unsigned h[kMaxBins + 2];
  for (int b = threadIdx.x; b <= kMaxBins + 1; b += blockDim.x) h[b] = 0;
  __syncthreads();
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n4;
       k += (int64_t)gridDim.x * blockDim.x) {
    const uint4 v = adj4[k];
    const uint32_t b[4] = {edge_bin(v.x), edge_bin(v.y), edge_bin(v.z), edge_bin(v.w)};
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (b[q] < (uint32_t)nb) atomicAdd(h + b[q], 1u);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nb; b += blockDim.x)
    if (h[b]) atomicAdd(pairs + b, (unsigned long long)h[b]);
}

// Weighted pair sums sum_{i<j} W_i W_j per bin (192-bit), and the weight
// moments sum W_i and sum W_i^2 (for the analytic random pair count).
__global__ void __launch_bounds__(kThreads) k_pairs_weighted(
    const int64_t* __restrict__ ptr, const int32_t* __restrict__ deg,
    const uint32_t* __restrict__ adj, int64_t adj_off, int64_t split, int64_t adj_off2,
    const int64_t* __restrict__ W, int64_t h0, int64_t h1, int nb, unsigned long long* pairs,
    unsigned long long* wpairs, unsigned long long* moments) {
  __shared__ unsigned long long acc[2 * (kMaxBins + 1)];
  __shared__ unsigned cnt[kMaxBins + 1];
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    acc[2 * b] = acc[2 * b + 1] = 0;
    cnt[b] = 0;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = h0 + blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < h1;
       i += warps) {
    const int64_t Wi = W[i];
    const int d = deg[i];
    const uint32_t* r = row_at(adj, ptr, i, adj_off, split, adj_off2);
    for (int k = lane; k < d; k += 32) {
      const uint32_t w = r[k];
      const int b = (int)edge_bin(w);
      long long lo, hi;
      mul_i128(Wi, W[edge_id(w)], &lo, &hi);
      atomic_add_i128(acc + 2 * b, lo, hi);
      atomicAdd(cnt + b, 1u);
    }
    if (lane == 0) {
      long long lo, hi;
      mul_i128(Wi, Wi, &lo, &hi);
      atomic_add_i192(moments + 3, (unsigned long long)lo, (unsigned long long)hi);
      atomic_add_i192(moments, (unsigned long long)Wi, (unsigned long long)(Wi < 0 ? -1ll : 0ll));
    }
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    if (acc[2 * b] | acc[2 * b + 1]) atomic_add_i192(wpairs + 3 * b, acc[2 * b], acc[2 * b + 1]);
    if (cnt[b]) atomicAdd(pairs + b, (unsigned long long)cnt[b]);
  }
}

__global__ void k_xi_disc(const unsigned long long* pairs, const double* wpairs_d,
                          const double* moments_d, const double* rr, const int64_t* e2g, int nb,
                          int64_t n, int64_t box, int weighted, double* xi_out,
                          const uint8_t* reps, int64_t n_orbits, double* zeta) {
  __shared__ double xi[kMaxBins + 1];
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    double RR;
    if (rr) {
      RR = rr[b];
    } else {
      double P;
      if (weighted) {
        const double S1 = moments_d[0], S2 = moments_d[1];
        P = __ddiv_rn(__dsub_rn(__dmul_rn(S1, S1), S2), 2.0);
      } else {
        P = __ddiv_rn(__dmul_rn((double)n, (double)(n - 1)), 2.0);
      }
      // edges from their squares (exact: the squares are perfect squares)
      const int64_t e0 = (int64_t)llrint(sqrt((double)e2g[b]));
      const int64_t e1 = (int64_t)llrint(sqrt((double)e2g[b + 1]));
      const double dv = (double)(e1 * e1 * e1 - e0 * e0 * e0);
      const double four_pi_3 = __ddiv_rn(__dmul_rn(4.0, 3.14159265358979323846), 3.0);
      const double vb = __dmul_rn(four_pi_3, dv);
      const double L = (double)box;
      const double vbox = __dmul_rn(__dmul_rn(L, L), L);
      RR = __ddiv_rn(__dmul_rn(P, vb), vbox);
    }
    const double num = weighted ? wpairs_d[b] : (double)pairs[b];
    const double x = __dsub_rn(__ddiv_rn(num, RR), 1.0);
    xi[b] = x;
    if (xi_out) xi_out[b] = x;
  }
  __syncthreads();
  if (!zeta) return;
  for (int64_t o = threadIdx.x; o < n_orbits; o += blockDim.x) {
    const uint8_t* r = reps + 6 * o;  // slots 01 02 03 12 13 23
    const double t1 = __dmul_rn(xi[r[0]], xi[r[5]]);
    const double t2 = __dmul_rn(xi[r[1]], xi[r[4]]);
    const double t3 = __dmul_rn(xi[r[2]], xi[r[3]]);
    zeta[o] = __dadd_rn(__dadd_rn(t1, t2), t3);
  }
}

}  // namespace

// Weighted pair sums of one graph: pairs[b] (counts), and on the device
// wp_d[0..nb) = sum_{i<j in bin b} w_i w_j, wp_d[nb] = sum w_i,
// wp_d[nb+1] = sum w_i^2, each the exact fixed-point sum rounded once.
int pairs_weighted_device(const Graph& g, const FixedW& fw, unsigned long long* pairs,
                          double* wp_d, const Opts& o, Scratch& sc, KernelTimer& timer) {
  cudaStream_t s = o.stream;
  const int nb = g.nb;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  unsigned long long* wacc = sc.alloc<unsigned long long>(3 * (size_t)nb + 6);
  if (!wacc) return GS_ENOMEM;
  cudaMemsetAsync(wacc, 0, sizeof(unsigned long long) * (3 * nb + 6), s);
  timer.start(s);
  int st = GS_OK;
  if (g.n)
    st = for_each_window(g, o, sc, [&](const WinView& v) -> int {
      { k_pairs_weighted<<<sms * 8, kThreads, 0, s>>>(g.d_ptr, g.d_deg, v.adj, v.off1, v.split, v.off2,
                                                    fw.d_W, v.h0, v.h1, nb, pairs, wacc,
                                                    wacc + 3 * nb); note_launch(); }
      return cuda_status(cudaGetLastError());
    });
  timer.stop(s);
  if (st) return st;
  { k_i192_to_double<<<1, 256, 0, s>>>(wacc, nb, 2 * fw.scale, wp_d); note_launch(); }
  { k_i192_to_double<<<1, 32, 0, s>>>(wacc + 3 * nb, 1, fw.scale, wp_d + nb); note_launch(); }
  { k_i192_to_double<<<1, 32, 0, s>>>(wacc + 3 * nb + 3, 1, 2 * fw.scale, wp_d + nb + 1); note_launch(); }
  return cuda_status(cudaGetLastError());
}

int pairs_disc_device(const Graph& g, const FixedW* fw, const double* d_rr, uint64_t* d_pairs,
                      double* d_xi, double* d_zeta, const Opts& o, Scratch& sc) {
  cudaStream_t s = o.stream;
  const int nb = g.nb;
  int st = GS_OK;
  const Conf4Tables* t = nullptr;
  if (d_zeta) {
    t = conf4_tables(nb, &st);
    if (!t) return st;
  }
  unsigned long long* pairs = d_pairs ? reinterpret_cast<unsigned long long*>(d_pairs)
                                      : sc.alloc<unsigned long long>(nb);
  if (!pairs) return GS_ENOMEM;
  cudaMemsetAsync(pairs, 0, sizeof(uint64_t) * nb, s);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  double* wp_d = nullptr;
  double* mom_d = nullptr;
  KernelTimer timer(o.kernel_ms);
  if (fw) {
    wp_d = sc.alloc<double>(nb + 2);
    if (!wp_d) return GS_ENOMEM;
    st = pairs_weighted_device(g, *fw, pairs, wp_d, o, sc, timer);
    if (st) return st;
    mom_d = wp_d + nb;
  } else if (g.slots) {
    timer.start(s);
    // the own rows of a window are its first ptr[h1] - ptr[h0] words
    st = for_each_window(g, o, sc, [&](const WinView& v) -> int {
      // the window's own rows are contiguous from row h0 (below any split)
      const int64_t words = g.h_ptr[v.h1] - g.h_ptr[v.h0];
      const uint32_t* own = v.adj + (g.h_ptr[v.h0] - v.off1);
      if (words)
        { k_pairs_count<<<sms * 8, kThreads, 0, s>>>(reinterpret_cast<const uint4*>(own), words / 4, nb,
                                                   pairs); note_launch(); }
      return cuda_status(cudaGetLastError());
    });
    timer.stop(s);
    if (st) return st;
  }
  if (d_xi || d_zeta) {
    { k_xi_disc<<<1, 1024, 0, s>>>(pairs, wp_d, mom_d, d_rr, g.d_edges2, nb, g.n, g.box_u, fw ? 1 : 0,
                                 d_xi, t ? t->d_reps : nullptr, t ? t->n_orbits : 0, d_zeta); note_launch(); }
  }
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e);
  timer.publish();
  return cuda_status(cudaGetLastError());
}

// Signed-weight estimator (Sec. 3.3): with data weights summing to +1 and
// random weights to -1 on the union, the signed pair sum is the
// Landy-Szalay numerator and xi = signed pair sum / RR needs no constant;
// zeta = signed quadruplet sum / RRRR per channel, and Eq. conn removes the
// disconnected part (Eq. disc, from this xi) from the even channel only.
// Every division and product is a single IEEE-rounded FP64 operation,
// left to right, no contraction.
__global__ void k_connected(const double* nn, const double* rr, const double* ne,
                            const double* no, const double* re, int nb, const uint8_t* reps,
                            int64_t n_orbits, double* xi_out, double* zeta_even,
                            double* zeta_odd, double* zeta_disc, double* zeta_conn) {
  __shared__ double xi[kMaxBins + 1];
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    xi[b] = __ddiv_rn(nn[b], rr[b]);
    if (xi_out) xi_out[b] = xi[b];
  }
  __syncthreads();
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n_orbits;
       o += (int64_t)gridDim.x * blockDim.x) {
    const uint8_t* r = reps + 6 * o;  // slots 01 02 03 12 13 23
    const double t1 = __dmul_rn(xi[r[0]], xi[r[5]]);
    const double t2 = __dmul_rn(xi[r[1]], xi[r[4]]);
    const double t3 = __dmul_rn(xi[r[2]], xi[r[3]]);
    const double disc = __dadd_rn(__dadd_rn(t1, t2), t3);
    const double ze = __ddiv_rn(ne[o], re[o]);
    if (zeta_even) zeta_even[o] = ze;
    if (zeta_odd) zeta_odd[o] = __ddiv_rn(no[o], re[o]);
    if (zeta_disc) zeta_disc[o] = disc;
    if (zeta_conn) zeta_conn[o] = __dsub_rn(ze, disc);
  }
}

int connected_device(const Graph& gdr, const FixedW& fdr, const Graph& gr, const FixedW& fr,
                     double* d_xi, double* d_even, double* d_odd, double* d_disc, double* d_conn,
                     const Opts& o, Scratch& sc) {
  cudaStream_t s = o.stream;
  const int nb = gdr.nb;
  int st = GS_OK;
  const Conf4Tables* t = conf4_tables(nb, &st);
  if (!t) return st;
  const int64_t no = t->n_orbits;
  unsigned long long* pairs = sc.alloc<unsigned long long>(2 * (size_t)nb);
  double* nn = sc.alloc<double>(nb + 2);
  double* rr = sc.alloc<double>(nb + 2);
  uint64_t* cnt = sc.alloc<uint64_t>(no);
  int64_t* odd = sc.alloc<int64_t>(no);
  double* ne = sc.alloc<double>(no);
  double* nodd = sc.alloc<double>(no);
  double* re = sc.alloc<double>(no);
  if (!pairs || !nn || !rr || !cnt || !odd || !ne || !nodd || !re) return GS_ENOMEM;
  cudaMemsetAsync(pairs, 0, sizeof(unsigned long long) * 2 * nb, s);
  // each pass reports its own kernel time; the call reports their sum
  double ms[4] = {0.0, 0.0, 0.0, 0.0};
  Opts sub = o;
  {
    KernelTimer timer(o.kernel_ms ? ms : nullptr);
    st = pairs_weighted_device(gdr, fdr, pairs, nn, o, sc, timer);
    if (!st) st = pairs_weighted_device(gr, fr, pairs + nb, rr, o, sc, timer);
    if (!st) st = cuda_status(cudaStreamSynchronize(s));
    if (st) return st;
    timer.publish();
  }
  sub.kernel_ms = o.kernel_ms ? ms + 1 : nullptr;
  st = count4_device(gdr, &fdr, true, cnt, odd, ne, nodd, sub, sc);
  if (st) return st;
  sub.kernel_ms = o.kernel_ms ? ms + 2 : nullptr;
  st = count4_device(gr, &fr, false, cnt, nullptr, re, nullptr, sub, sc);
  if (st) return st;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = (int)std::min<int64_t>(sms, (no + 255) / 256);
  { k_connected<<<std::max(blocks, 1), 256, 0, s>>>(nn, rr, ne, nodd, re, nb, t->d_reps, no, d_xi, d_even,
                                                  d_odd, d_disc, d_conn); note_launch(); }
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e);
  if (o.kernel_ms) *o.kernel_ms = ms[0] + ms[1] + ms[2];
  return cuda_status(cudaGetLastError());
}

}  // namespace gs
