// Internal declarations of the GB300 query engine (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "../../include/gramsci_gb300.h"

namespace gs {

// ----------------------------------------------------------------------------
// Edge storage. Every stored edge is one 32-bit word (neighbour id << 8 | bin),
// so a row sorted by word is sorted by neighbour id, one 128-bit load brings
// four edges, and a bin costs no separate array. Rows start on a multiple of
// four words (16 bytes, the bulk-copy alignment) and are padded with
// kSentinel, whose id field (2^24 - 1) exceeds every real id (n < 2^24).
constexpr uint32_t kSentinel = 0xFFFFFFFFu;
constexpr int kRowAlign = 4;
constexpr int64_t kMaxPoints = (int64_t(1) << 24) - 1;
constexpr int kMaxBins = 254;
constexpr int kMaxBins4 = 16;

__host__ __device__ inline uint32_t edge_id(uint32_t w) { return w >> 8; }
__host__ __device__ inline uint32_t edge_bin(uint32_t w) { return w & 0xFFu; }
__host__ __device__ inline int64_t pad_row(int64_t d) {
  return (d + kRowAlign - 1) / kRowAlign * kRowAlign;
}

// Device-wide error flags written by kernels, read by the host after a sync.
enum : int { kErrNone = 0, kErrTimeout = 1, kErrRange = 2, kErrOverflow = 4 };

// Process-wide count of kernel launches made by the library.
void note_launch();

// Device time of selected launches, measured with CUDA events on the
// launch stream; the sum is read after the stream has been synchronised.
class KernelTimer {
 public:
  explicit KernelTimer(double* out) : out_(out) {}
  ~KernelTimer();
  void start(cudaStream_t s);
  void stop(cudaStream_t s);
  void publish();  // call after the stream is synchronised

 private:
  double* out_;
  std::vector<cudaEvent_t> ev_;
};

struct Graph {
  int64_t n = 0;
  int nb = 0;
  int64_t box_u = 0;
  std::vector<int64_t> edges;  // nb+1 lattice-unit bin edges (host)
  int64_t* d_edges2 = nullptr;  // nb+1 squared edges (device)
  int4* d_xyzp = nullptr;       // [n] (x, y, z, caller index) in internal order
  int32_t* d_deg = nullptr;     // [n] |N+(i)|
  int64_t* d_ptr = nullptr;     // [n+1] row starts (words)
  uint32_t* d_adj = nullptr;    // [slots] packed edge words (resident graphs)
  uint32_t* h_adj = nullptr;    // [slots] pinned host copy (out-of-core graphs)
  std::vector<int64_t> h_ptr;   // host copy of d_ptr (window planning)
  std::vector<int32_t> h_deg;   // host copy of d_deg
  // out-of-core planning. In a periodic box the ids are x-major, so hubs
  // of the first x-slab have wrap-around neighbours in the last one:
  // wrap_start is the first id of the last x-slab (n for an open box);
  // h_reach[i] is the largest neighbour id of i below wrap_start (or i) and
  // h_far[i] says whether i has neighbours at or above wrap_start.
  std::vector<int32_t> h_reach;
  std::vector<uint8_t> h_far;
  int64_t wrap_start = 0;
  int64_t slots = 0;
  int64_t edges_total = 0;
  int64_t probe_words = 0;
  int64_t walk_words = -1;  // computed on first request
  int max_deg = 0;
  int cells[3] = {0, 0, 0};
  int windows = 1;
  uint64_t budget = 0;     // build-time device budget (default for queries)
  int force_windows = 0;   // build-time forced window count (default for queries)
  int64_t device_bytes = 0;
  int device = 0;
};

// Options with defaults applied.
struct Opts {
  uint64_t budget = 0;
  int force_windows = 0;
  int variant = 0;
  cudaStream_t stream = nullptr;
  double* kernel_ms = nullptr;
  int shard = 0, shards = 0;
};

// Hub range [lo, hi) of the query's shard (the whole graph when unsharded).
void shard_range(const Graph& g, const Opts& o, int64_t* lo, int64_t* hi);
Opts read_opts(const gs_options* o);

// Whether p is device-accessible memory of the current device.
bool is_device_ptr(const void* p);

// Stream-ordered scratch allocations released at scope exit.
class Scratch {
 public:
  explicit Scratch(cudaStream_t s) : s_(s) {}
  ~Scratch();
  template <class T>
  T* alloc(size_t count) {
    return static_cast<T*>(alloc_bytes(count * sizeof(T)));
  }
  void* alloc_bytes(size_t bytes);
  bool failed() const { return failed_; }

 private:
  cudaStream_t s_;
  std::vector<void*> ptrs_;
  bool failed_ = false;
};

// Copy a caller array to the device when it lives on the host; returns a
// device pointer (the caller's own when already on the device).
const void* to_device(Scratch& sc, const void* p, size_t bytes, cudaStream_t s);

// Status from a CUDA error.
int cuda_status(cudaError_t e);

// Exclusive scans (device, stream ordered). out may alias in.
int scan_exclusive_i32(const int32_t* in, int32_t* out, int64_t n, int32_t* total_dev,
                       cudaStream_t s, Scratch& sc);
int scan_exclusive_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s, Scratch& sc);

// Configuration tables (host-built, cached per nb).
struct Conf4Tables {
  int nb = 0;
  int64_t n_orbits = 0;
  // raw tuple index with digit order (b01, b02, b12, b03, b13, b23), most
  // significant first -> orbit | (odd relabelling) << 30 | chiral << 31
  std::vector<uint32_t> lut;
  std::vector<uint8_t> reps;    // n_orbits * 6 in slot order (01,02,03,12,13,23)
  std::vector<uint8_t> chiral;  // n_orbits
  uint32_t* d_lut = nullptr;
  uint8_t* d_reps = nullptr;
  int device = -1;
};
const Conf4Tables* conf4_tables(int nb, int* status);  // host tables + device copy
const Conf4Tables* conf4_host(int nb, int* status);    // host tables only
int64_t num_conf3(int nb);

// Fixed-point weights: W_i = w_i * 2^scale is an integer for every point.
struct FixedW {
  int64_t* d_W = nullptr;  // [n], internal order
  int scale = 0;
  int bits = 0;  // max bit length of |W_i| plus one sign bit
  bool nonneg = true;  // no weight is negative
};
// max_bits: the widest |W| (bits, sign included) the caller can sum exactly:
// 31 for the kernels' direct path, up to 54 where the caller splits wide
// weights (below); wider weights give GS_EUNSUPPORTED.
int prepare_weights(const Graph& g, const float* w, FixedW* out, Scratch& sc, cudaStream_t s,
                    int max_bits = 31);
constexpr int kNarrowWeightBits = 31;

// Wide weights (csrc/gs_wide.cu): out = A + t B with W = A + 2^27 B,
// 0 <= A < 2^27; and the exact interpolation of degree-3 or degree-4 sums
// evaluated at t = 0, 1, -1, 2[, -2] (blocks of n 192-bit sums in d_P), at
// t = 2^27, rounded once to double with the given scale.
int split_weights_device(const FixedW& fw, int64_t n, int t, int64_t* d_out, cudaStream_t s);
int combine_wide_device(const unsigned long long* d_P, int64_t n, int degree, int scale,
                        double* d_out, cudaStream_t s);
int wide_eval_point(int k);

// Kernel launchers (defined in the per-stage .cu files).
int build_graph_device(const int32_t* d_xyz, int64_t n, int64_t box_u,
                       const std::vector<int64_t>& edges, const Opts& o, Graph* g);
// equi: the equilateral configurations (b, b, b) only, nb outputs.
// wacc_out: NULL, or n_conf 192-bit accumulators that receive the exact
// weighted sums (zeroed here) instead of a rounded d_wsum.
int count3_device(const Graph& g, const FixedW* fw, uint64_t* d_counts, double* d_wsum,
                  const Opts& o, Scratch& sc, bool equi = false,
                  unsigned long long* wacc_out = nullptr);
// Anisotropic 3pCF (csrc/gs_mu.cu): counts [nconf][nmu + 1] by configuration
// and mu bin of the triangle's normal against the z axis (bin nmu:
// collinear); d_wsum NULL or the same shape (narrow weights only).
int count3mu_device(const Graph& g, const FixedW* fw, int nmu, uint64_t* d_counts,
                    double* d_wsum, const Opts& o, Scratch& sc);
int count3_batch_device(const Graph* const* gr, int ng, const FixedW* fws, uint64_t* const* d_counts,
                        double* const* d_wsum, const Opts& o, Scratch& sc);
// pix: the odd channel from pixelised spoke directions (parity only)
int count4_device(const Graph& g, const FixedW* fw, bool parity, uint64_t* d_even,
                  int64_t* d_odd, double* d_weven, double* d_wodd, const Opts& o, Scratch& sc,
                  bool pix = false, unsigned long long* weven_out = nullptr,
                  unsigned long long* wodd_out = nullptr);
int direction_pixels_device(const int32_t* d_dirs, int64_t n, uint8_t* d_out, cudaStream_t s);
int pairs_disc_device(const Graph& g, const FixedW* fw, const double* d_rr, uint64_t* d_pairs,
                      double* d_xi, double* d_zeta, const Opts& o, Scratch& sc);
int connected_device(const Graph& gdr, const FixedW& fdr, const Graph& gr, const FixedW& fr,
                     double* d_xi, double* d_even, double* d_odd, double* d_disc, double* d_conn,
                     const Opts& o, Scratch& sc);
int walk_words_device(Graph* g);
int tri_words_device(const Graph& g, int64_t* tri, int64_t* words);
int quantize_device(const double* d_pos, int64_t n, int64_t box_u, int periodic, int32_t* d_xyz,
                    cudaStream_t s, Scratch& sc);

// ----------------------------------------------------------------------------
// Out-of-core row windows. Window k covers hubs [h0, h1). The rows it needs
// (the hubs' own rows and every spoke row) are at most two id ranges,
// because every spoke id is above its hub: [h0, r1) with r1 = 1 + the
// largest neighbour id below wrap_start, plus [wrap_start, n) when a hub
// has wrap-around neighbours. Each hub belongs to exactly one window, so
// every tuple is counted exactly once.
struct WindowPlan {
  std::vector<int64_t> h0, h1, r1;
  std::vector<uint8_t> far;  // the window also needs rows [wrap_start, n)
  int64_t max_words = 0;
};
int plan_windows(const Graph& g, const Opts& o, WindowPlan* plan, int64_t lo, int64_t hi);

// Where the rows of one window live: row j starts at
// adj + ptr[j] - (j >= split ? off2 : off1).
struct WinView {
  const uint32_t* adj;
  int64_t off1, split, off2;
  int64_t h0, h1;
};

__host__ __device__ inline const uint32_t* row_at(const uint32_t* adj, const int64_t* ptr,
                                                  int64_t j, int64_t off1, int64_t split,
                                                  int64_t off2) {
  return adj + (ptr[j] - (j >= split ? off2 : off1));
}

// Streams the windows of an out-of-core graph through two device buffers:
// the copy of window k+1 (pinned host -> device, on a side stream) overlaps
// the counting of window k on o.stream. fn(const WinView&) launches the
// counting of the window's hubs. A resident graph makes one call with its
// own edge array.
template <class F>
int for_each_window(const Graph& g, const Opts& o, Scratch& sc, F&& fn) {
  int64_t lo = 0, hi = 0;
  shard_range(g, o, &lo, &hi);
  if (lo >= hi) return GS_OK;
  if (g.d_adj) {
    const WinView v{g.d_adj, 0, g.n, 0, lo, hi};
    return fn(v);
  }
  WindowPlan plan;
  int st = plan_windows(g, o, &plan, lo, hi);
  if (st) return st;
  const size_t nw = plan.h0.size();
  uint32_t* buf[2] = {sc.alloc<uint32_t>(plan.max_words),
                      nw > 1 ? sc.alloc<uint32_t>(plan.max_words) : nullptr};
  if (!buf[0] || (nw > 1 && !buf[1])) return GS_ENOMEM;
  cudaStream_t cs = nullptr;
  cudaEvent_t ready = nullptr, copied[2] = {nullptr, nullptr}, done[2] = {nullptr, nullptr};
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ready, cudaEventDisableTiming);
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
    e = cudaEventCreateWithFlags(&copied[b], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&done[b], cudaEventDisableTiming);
  }
  const int64_t n = g.n;
  if (e == cudaSuccess) {
    // the buffers were allocated in o.stream's order
    cudaEventRecord(ready, o.stream);
    cudaStreamWaitEvent(cs, ready, 0);
    for (size_t k = 0; k < nw && !st; ++k) {
      const int b = (int)(k & 1);
      if (k >= 2) cudaStreamWaitEvent(cs, done[b], 0);
      const int64_t off1 = g.h_ptr[plan.h0[k]];
      const int64_t len1 = g.h_ptr[plan.r1[k]] - off1;
      e = cudaMemcpyAsync(buf[b], g.h_adj + off1, sizeof(uint32_t) * len1, cudaMemcpyHostToDevice,
                          cs);
      WinView v{buf[b], off1, n, 0, plan.h0[k], plan.h1[k]};
      if (e == cudaSuccess && plan.far[k]) {
        const int64_t w0 = g.h_ptr[g.wrap_start];
        e = cudaMemcpyAsync(buf[b] + len1, g.h_adj + w0, sizeof(uint32_t) * (g.h_ptr[n] - w0),
                            cudaMemcpyHostToDevice, cs);
        v.split = g.wrap_start;
        v.off2 = w0 - len1;
      }
      if (e != cudaSuccess) break;
      cudaEventRecord(copied[b], cs);
      cudaStreamWaitEvent(o.stream, copied[b], 0);
      st = fn(v);
      cudaEventRecord(done[b], o.stream);
    }
    cudaStreamSynchronize(cs);
  }
  if (!st && e != cudaSuccess) st = cuda_status(e);
  for (int b = 0; b < 2; ++b) {
    if (copied[b]) cudaEventDestroy(copied[b]);
    if (done[b]) cudaEventDestroy(done[b]);
  }
  if (ready) cudaEventDestroy(ready);
  if (cs) cudaStreamDestroy(cs);
  return st;
}

// Device helpers shared by the counting kernels --------------------------------

// 128-bit two's-complement accumulation into (lo, hi) words with carry.
__device__ inline void atomic_add_i128(unsigned long long* lo_hi, long long plo_s,
                                       long long phi_s) {
  const unsigned long long plo = (unsigned long long)plo_s;
  const unsigned long long phi = (unsigned long long)phi_s;
  const unsigned long long old = atomicAdd(lo_hi, plo);
  const unsigned long long carry = (old + plo < old) ? 1ull : 0ull;
  if (phi + carry) atomicAdd(lo_hi + 1, phi + carry);
}

// 192-bit accumulation (three limbs) of a 128-bit signed value.
__device__ inline void atomic_add_i192(unsigned long long* limbs, unsigned long long lo,
                                       unsigned long long hi) {
  const unsigned long long ext = ((long long)hi < 0) ? ~0ull : 0ull;
  const unsigned long long o0 = atomicAdd(limbs, lo);
  const unsigned long long c0 = (o0 + lo < o0) ? 1ull : 0ull;
  const unsigned long long add1 = hi + c0;
  const unsigned long long c1a = (add1 < hi) ? 1ull : 0ull;  // hi + c0 wrapped
  const unsigned long long o1 = atomicAdd(limbs + 1, add1);
  const unsigned long long c1b = (o1 + add1 < o1) ? 1ull : 0ull;
  const unsigned long long add2 = ext + c1a + c1b;
  if (add2) atomicAdd(limbs + 2, add2);
}

// Signed 64 x 64 -> 128-bit product as (lo, hi).
__device__ inline void mul_i128(long long a, long long b, long long* lo, long long* hi) {
  *lo = (long long)((unsigned long long)a * (unsigned long long)b);
  *hi = __mul64hi(a, b);
}

// An integer below 2^40 in magnitude to the nearest float without a 64-bit
// integer conversion (on GB300 those run on the slow FP64 pipe): v = hi 2^16
// + lo with 0 <= lo < 2^16, both halves convert exactly, and the fused
// multiply-add rounds the exact sum once.
__device__ inline float i40_to_float(long long v) {
  const int hi = (int)(v >> 16), lo = (int)(v & 0xFFFF);
  return fmaf((float)hi, 65536.0f, (float)lo);
}

// Canonical rank of the sorted bin triple of (x, y, z), Sec. 5.1 ordering.
__device__ __host__ inline int conf3_rank(int x, int y, int z, int nb) {
  int a = x < y ? x : y, b = x < y ? y : x;
  int c = z;
  if (c < b) {
    int t = b;
    b = c;
    c = t;
    if (b < a) {
      t = a;
      a = b;
      b = t;
    }
  }
  // triples with first < a: H(nb) - H(nb - a), H(k) = k(k+1)(k+2)/6
  const int ka = nb - a;
  const int first = (nb * (nb + 1) * (nb + 2) - ka * (ka + 1) * (ka + 2)) / 6;
  const int second = (b - a) * nb - ((a + b - 1) * (b - a)) / 2;
  return first + second + (c - b);
}

// Bounded spin: returns false after `limit` failed polls of an mbarrier phase.
__device__ inline bool mbar_wait(uint64_t* bar, uint32_t phase, uint32_t limit) {
  const uint32_t addr = (uint32_t)__cvta_generic_to_shared(bar);
  for (uint32_t it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(addr), "r"(phase)
        : "memory");
    if (done) return true;
    if (it > 64) __nanosleep(32);
  }
  return false;
}

__device__ inline void mbar_init(uint64_t* bar, uint32_t count) {
  const uint32_t addr = (uint32_t)__cvta_generic_to_shared(bar);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One-dimensional bulk copy global -> shared (TMA engine, no tensor map),
// completing on `bar` with `bytes` of transaction count. Both addresses must
// be 16-byte aligned and bytes a multiple of 16.
__device__ inline void bulk_load(void* smem_dst, const void* gmem_src, uint32_t bytes,
                                 uint64_t* bar) {
  const uint32_t dst = (uint32_t)__cvta_generic_to_shared(smem_dst);
  const uint32_t b = (uint32_t)__cvta_generic_to_shared(bar);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(gmem_src), "r"(bytes), "r"(b)
      : "memory");
}

// Asynchronous 16-byte global -> shared copies (cp.async, L2 only). The
// source and destination must be 16-byte aligned. Groups are per thread:
// commit closes the thread's current group, wait<N> returns when at most N
// of the thread's groups are still in flight.
__device__ inline void cp_async16(void* smem_dst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ inline void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
__device__ inline void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ inline uint4 ldg_nc_v4(const uint32_t* p) {
  uint4 v;
  asm volatile("ld.global.nc.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}

constexpr uint32_t kHashMul = 2654435761u;  // Knuth's multiplicative constant
constexpr uint32_t kWaitLimit = 1u << 24;   // polls before a wait gives up

}  // namespace gs

struct gs_graph {
  gs::Graph g;
};
struct gs_plan;
