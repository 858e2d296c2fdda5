// C ABI entry points, host orchestration and shared host utilities.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>

#include "gs_internal.cuh"

namespace gs {

Opts read_opts(const gs_options* o) {
  Opts r;
  if (o) {
    r.budget = o->device_budget_bytes;
    r.force_windows = o->force_windows;
    r.variant = o->variant;
    r.stream = static_cast<cudaStream_t>(o->stream);
    r.kernel_ms = o->kernel_ms;
    r.shard = o->shard;
    r.shards = o->shards;
  }
  return r;
}

namespace {
std::atomic<unsigned long long> g_launches{0};
}
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

KernelTimer::~KernelTimer() {
  for (cudaEvent_t e : ev_) cudaEventDestroy(e);
}
void KernelTimer::start(cudaStream_t s) {
  if (!out_) return;
  cudaEvent_t e;
  if (cudaEventCreate(&e) != cudaSuccess) return;
  cudaEventRecord(e, s);
  ev_.push_back(e);
}
void KernelTimer::stop(cudaStream_t s) { start(s); }
void KernelTimer::publish() {
  if (!out_) return;
  double ms = 0.0;
  for (size_t k = 0; k + 1 < ev_.size(); k += 2) {
    float f = 0.f;
    if (cudaEventElapsedTime(&f, ev_[k], ev_[k + 1]) == cudaSuccess) ms += f;
  }
  *out_ = ms;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return GS_OK;
  if (e == cudaErrorMemoryAllocation) return GS_ENOMEM;
  return GS_ECUDA;
}

Scratch::~Scratch() {
  for (void* p : ptrs_) cudaFreeAsync(p, s_);
}

void* Scratch::alloc_bytes(size_t bytes) {
  if (bytes == 0) bytes = 16;
  void* p = nullptr;
  if (cudaMallocAsync(&p, bytes, s_) != cudaSuccess) {
    cudaGetLastError();
    failed_ = true;
    return nullptr;
  }
  ptrs_.push_back(p);
  return p;
}

const void* to_device(Scratch& sc, const void* p, size_t bytes, cudaStream_t s) {
  if (!p) return nullptr;
  if (is_device_ptr(p)) return p;
  void* d = sc.alloc_bytes(bytes);
  if (!d) return nullptr;
  if (cudaMemcpyAsync(d, p, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) return nullptr;
  return d;
}

// ----------------------------------------------------------------------------
// Exclusive scan: per-block totals, recursive scan of the totals, per-block
// scan with the block offset. 1024 threads x 4 items per block.
namespace {
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

template <class T>
__device__ T block_exclusive_scan(T v, T* total) {
  __shared__ T warp_sums[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  T x = v;
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[wid] = x;
  __syncthreads();
  if (wid == 0) {
    T s = (lane < (int)(blockDim.x >> 5)) ? warp_sums[lane] : T(0);
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    warp_sums[lane] = s;
  }
  __syncthreads();
  const T warp_off = wid ? warp_sums[wid - 1] : T(0);
  *total = warp_sums[(blockDim.x >> 5) - 1];
  __syncthreads();
  return warp_off + x - v;
}

template <class T>
__global__ void k_scan_block_totals(const T* in, int64_t n, T* totals) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  T s = 0;
  for (int k = 0; k < kScanItems; ++k)
    if (base + k < n) s += in[base + k];
  T tot;
  block_exclusive_scan<T>(s, &tot);
  if (threadIdx.x == 0) totals[blockIdx.x] = tot;
}

template <class T>
__global__ void k_scan_apply(const T* in, T* out, int64_t n, const T* offsets, T* grand_total) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  T v[kScanItems];
  T s = 0;
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = (base + k < n) ? in[base + k] : T(0);
    s += v[k];
  }
  T tot;
  T run = block_exclusive_scan<T>(s, &tot) + (offsets ? offsets[blockIdx.x] : T(0));
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
  if (grand_total && blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1)
    *grand_total = run;
}

template <class T>
int scan_impl(const T* in, T* out, int64_t n, T* total_dev, cudaStream_t s, Scratch& sc) {
  if (n <= 0) {
    if (total_dev) cudaMemsetAsync(total_dev, 0, sizeof(T), s);
    return GS_OK;
  }
  const int64_t blocks = (n + kScanTile - 1) / kScanTile;
  if (blocks == 1) {
    { k_scan_apply<T><<<1, kScanThreads, 0, s>>>(in, out, n, nullptr, total_dev); note_launch(); }
    return cuda_status(cudaGetLastError());
  }
  T* totals = sc.alloc<T>(blocks);
  if (!totals) return GS_ENOMEM;
  { k_scan_block_totals<T><<<(unsigned)blocks, kScanThreads, 0, s>>>(in, n, totals); note_launch(); }
  int st = scan_impl<T>(totals, totals, blocks, nullptr, s, sc);
  if (st) return st;
  { k_scan_apply<T><<<(unsigned)blocks, kScanThreads, 0, s>>>(in, out, n, totals, total_dev); note_launch(); }
  return cuda_status(cudaGetLastError());
}
}  // namespace

int scan_exclusive_i32(const int32_t* in, int32_t* out, int64_t n, int32_t* total_dev,
                       cudaStream_t s, Scratch& sc) {
  return scan_impl<int32_t>(in, out, n, total_dev, s, sc);
}
int scan_exclusive_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s, Scratch& sc) {
  return scan_impl<int64_t>(in, out, n, nullptr, s, sc);
}

// ----------------------------------------------------------------------------
// Configuration tables. The 4-point tables enumerate every raw edge-bin
// tuple, take the smallest of its 24 vertex relabellings as the canonical
// representative (Sec. 5.2) and rank representatives lexicographically.
int64_t num_conf3(int nb) { return (int64_t)nb * (nb + 1) * (nb + 2) / 6; }

namespace {
// For each vertex permutation p (new vertex k = old vertex p[k]) the slot
// of the new tuple that takes each old slot, for slots (01,02,03,12,13,23).
struct SlotPerms {
  int src[24][6];  // new slot s reads old slot src[p][s]
  int odd[24];
  SlotPerms() {
    static const int va[6] = {0, 0, 0, 1, 1, 2}, vb[6] = {1, 2, 3, 2, 3, 3};
    int p[4] = {0, 1, 2, 3};
    int q = 0;
    do {
      int inv = 0;
      for (int a = 0; a < 4; ++a)
        for (int b = a + 1; b < 4; ++b) inv += p[a] > p[b];
      odd[q] = inv & 1;
      for (int s = 0; s < 6; ++s) {
        int x = p[va[s]], y = p[vb[s]];
        if (x > y) std::swap(x, y);
        for (int t = 0; t < 6; ++t)
          if (va[t] == x && vb[t] == y) src[q][s] = t;
      }
      ++q;
    } while (std::next_permutation(p, p + 4));
  }
};

std::mutex g_conf_mu;
std::map<int, Conf4Tables*> g_conf4;
}  // namespace

// Host tables only (no CUDA call); the caller holds g_conf_mu.
static Conf4Tables* conf4_host_locked(int nb, int* status) {
  *status = GS_OK;
  if (nb < 1 || nb > kMaxBins4) {
    *status = GS_ERANGE;
    return nullptr;
  }
  auto it = g_conf4.find(nb);
  Conf4Tables* t = nullptr;
  if (it != g_conf4.end()) {
    t = it->second;
  } else {
    t = new (std::nothrow) Conf4Tables();
    if (!t) {
      *status = GS_ENOMEM;
      return nullptr;
    }
    static const SlotPerms P;
    t->nb = nb;
    const uint64_t NB = (uint64_t)nb;
    const uint64_t total = NB * NB * NB * NB * NB * NB;
    // Encode a tuple lexicographically in slot order (01,02,03,12,13,23).
    auto enc = [&](const int* tup) {
      uint64_t x = 0;
      for (int s = 0; s < 6; ++s) x = x * NB + (uint64_t)tup[s];
      return x;
    };
    std::vector<uint32_t> canon(total);   // lexicographic code of the representative
    std::vector<uint8_t> rel_odd(total);  // a minimising relabelling is odd
    std::vector<uint8_t> is_rep(total, 0);
    int tup[6], r[6];
    for (uint64_t code = 0; code < total; ++code) {
      uint64_t c = code;
      for (int s = 5; s >= 0; --s) {
        tup[s] = (int)(c % NB);
        c /= NB;
      }
      uint64_t best = code;
      int best_odd = 0;
      for (int q = 1; q < 24; ++q) {
        for (int s = 0; s < 6; ++s) r[s] = tup[P.src[q][s]];
        const uint64_t e = enc(r);
        if (e < best) {
          best = e;
          best_odd = P.odd[q];
        }
      }
      canon[code] = (uint32_t)best;
      rel_odd[code] = (uint8_t)best_odd;
      if (best == code) is_rep[code] = 1;
    }
    std::vector<int32_t> rank(total, -1);
    int64_t k = 0;
    for (uint64_t code = 0; code < total; ++code)
      if (is_rep[code]) rank[code] = (int32_t)k++;
    t->n_orbits = k;
    t->reps.resize((size_t)k * 6);
    t->chiral.assign((size_t)k, 1);
    for (uint64_t code = 0; code < total; ++code) {
      if (!is_rep[code]) continue;
      const int32_t o = rank[code];
      uint64_t c = code;
      for (int s = 5; s >= 0; --s) {
        tup[s] = (int)(c % NB);
        c /= NB;
      }
      for (int s = 0; s < 6; ++s) t->reps[(size_t)o * 6 + s] = (uint8_t)tup[s];
      for (int q = 1; q < 24; ++q) {
        if (!P.odd[q]) continue;
        for (int s = 0; s < 6; ++s) r[s] = tup[P.src[q][s]];
        if (enc(r) == code) t->chiral[o] = 0;
      }
    }
    // Device LUT in the kernels' digit order (b01, b02, b12, b03, b13, b23).
    t->lut.resize(total);
    for (uint64_t code = 0; code < total; ++code) {
      uint64_t c = code;
      for (int s = 5; s >= 0; --s) {
        tup[s] = (int)(c % NB);
        c /= NB;
      }
      const int kd[6] = {tup[0], tup[1], tup[3], tup[2], tup[4], tup[5]};
      uint64_t kidx = 0;
      for (int s = 0; s < 6; ++s) kidx = kidx * NB + (uint64_t)kd[s];
      const int32_t o = rank[canon[code]];
      t->lut[kidx] = (uint32_t)o | ((uint32_t)rel_odd[code] << 30) |
                     ((uint32_t)t->chiral[o] << 31);
    }
    g_conf4[nb] = t;
  }
  return t;
}

const Conf4Tables* conf4_host(int nb, int* status) {
  std::lock_guard<std::mutex> lock(g_conf_mu);
  return conf4_host_locked(nb, status);
}

const Conf4Tables* conf4_tables(int nb, int* status) {
  std::lock_guard<std::mutex> lock(g_conf_mu);
  Conf4Tables* t = conf4_host_locked(nb, status);
  if (!t) return nullptr;
  int dev = 0;
  cudaGetDevice(&dev);
  if (t->device != dev || !t->d_lut) {
    // (re)upload for the current device; the previous copy is left to the
    // process exit when several devices are used in turn
    uint32_t* dl = nullptr;
    uint8_t* dr = nullptr;
    cudaError_t e = cudaMalloc(&dl, t->lut.size() * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&dr, t->reps.size());
    if (e == cudaSuccess)
      e = cudaMemcpy(dl, t->lut.data(), t->lut.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dr, t->reps.data(), t->reps.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaGetLastError();
      if (dl) cudaFree(dl);
      if (dr) cudaFree(dr);
      *status = cuda_status(e);
      return nullptr;
    }
    t->d_lut = dl;
    t->d_reps = dr;
    t->device = dev;
  }
  return t;
}

// ----------------------------------------------------------------------------
// Weights: exact fixed point. For FP32 inputs with frexp exponents in
// [emin, emax], W_i = w_i * 2^(24 - emin) is an integer of at most
// 25 + (emax - emin) bits.
namespace {
__global__ void k_weight_exponents(const float* w, int64_t n, int* emin, int* emax, int* bad,
                                   int* neg) {
  int lo = 1 << 20, hi = -(1 << 20), b = 0, ng = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float x = w[i];
    if (!isfinite(x)) {
      b = 1;
      continue;
    }
    if (x < 0.0f) ng = 1;
    if (x == 0.0f) continue;
    int e;
    frexpf(x, &e);
    lo = min(lo, e);
    hi = max(hi, e);
  }
  for (int o = 16; o; o >>= 1) {
    lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    b |= __shfl_xor_sync(0xffffffffu, b, o);
    ng |= __shfl_xor_sync(0xffffffffu, ng, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(emin, lo);
    atomicMax(emax, hi);
    if (b) atomicOr(bad, 1);
    if (ng) atomicOr(neg, 1);
  }
}

__global__ void k_weight_fixed(const float* w, const int4* xyzp, int64_t n, int scale,
                               int64_t* W) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float x = w[xyzp[i].w];
    W[i] = (int64_t)ldexp((double)x, scale);  // exact: x * 2^scale is an integer
  }
}
}  // namespace

int prepare_weights(const Graph& g, const float* w, FixedW* out, Scratch& sc, cudaStream_t s,
                    int max_bits) {
  const float* dw = static_cast<const float*>(to_device(sc, w, sizeof(float) * g.n, s));
  int* flags = sc.alloc<int>(4);
  int64_t* W = sc.alloc<int64_t>(g.n);
  if (!dw || !flags || !W) return GS_ENOMEM;
  const int init[4] = {1 << 20, -(1 << 20), 0, 0};
  cudaMemcpyAsync(flags, init, sizeof(init), cudaMemcpyHostToDevice, s);
  { k_weight_exponents<<<304, 256, 0, s>>>(dw, g.n, flags, flags + 1, flags + 2, flags + 3); note_launch(); }
  int h[4];
  cudaMemcpyAsync(h, flags, sizeof(h), cudaMemcpyDeviceToHost, s);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e);
  if (h[2]) return GS_EUNSUPPORTED;
  if (h[0] > h[1]) h[0] = h[1] = 0;  // all weights zero
  out->scale = 24 - h[0];
  out->bits = 25 + (h[1] - h[0]) + 1;
  out->nonneg = h[3] == 0;
  if (out->bits > max_bits) return GS_EUNSUPPORTED;
  { k_weight_fixed<<<304, 256, 0, s>>>(dw, g.d_xyzp, g.n, out->scale, W); note_launch(); }
  out->d_W = W;
  return cuda_status(cudaGetLastError());
}

// Wide weights: the sums of degree-3 (triangles) or degree-4 (tetrahedra)
// weight products evaluated exactly at t = 0, 1, -1, 2[, -2] on the split
// weights A + t B, then interpolated and rounded once (csrc/gs_wide.cu).
int count3_wide(const Graph& g, const FixedW& fw, uint64_t* d_counts, double* d_wsum,
                const Opts& o, Scratch& sc) {
  const int64_t nc = num_conf3(g.nb);
  const int npts = 4;
  unsigned long long* P = sc.alloc<unsigned long long>(3 * (size_t)nc * npts);
  int64_t* Wt = sc.alloc<int64_t>(g.n > 0 ? g.n : 1);
  if (!P || !Wt) return GS_ENOMEM;
  FixedW ft;
  ft.d_W = Wt;
  ft.scale = fw.scale;
  ft.bits = 30;
  ft.nonneg = false;
  int st = GS_OK;
  for (int k = 0; k < npts && !st; ++k) {
    st = split_weights_device(fw, g.n, wide_eval_point(k), Wt, o.stream);
    if (!st) st = count3_device(g, &ft, d_counts, nullptr, o, sc, false, P + 3 * (size_t)nc * k);
  }
  if (!st) st = combine_wide_device(P, nc, 3, 3 * fw.scale, d_wsum, o.stream);
  return st;
}

int count4_wide(const Graph& g, const FixedW& fw, bool parity, bool pix, uint64_t* d_even,
                int64_t* d_odd, double* d_weven, double* d_wodd, const Opts& o, Scratch& sc) {
  int st = GS_OK;
  const Conf4Tables* t = conf4_tables(g.nb, &st);
  if (!t) return st;
  const int64_t no = t->n_orbits;
  const int npts = 5;
  unsigned long long* Pe = sc.alloc<unsigned long long>(3 * (size_t)no * npts);
  unsigned long long* Po = parity ? sc.alloc<unsigned long long>(3 * (size_t)no * npts) : nullptr;
  int64_t* Wt = sc.alloc<int64_t>(g.n > 0 ? g.n : 1);
  if (!Pe || (parity && !Po) || !Wt) return GS_ENOMEM;
  FixedW ft;
  ft.d_W = Wt;
  ft.scale = fw.scale;
  ft.bits = 30;
  ft.nonneg = false;
  for (int k = 0; k < npts && !st; ++k) {
    st = split_weights_device(fw, g.n, wide_eval_point(k), Wt, o.stream);
    if (!st)
      st = count4_device(g, &ft, parity, d_even, d_odd, nullptr, nullptr, o, sc, pix,
                         Pe + 3 * (size_t)no * k, parity ? Po + 3 * (size_t)no * k : nullptr);
  }
  if (!st && d_weven) st = combine_wide_device(Pe, no, 4, 4 * fw.scale, d_weven, o.stream);
  if (!st && d_wodd && parity) st = combine_wide_device(Po, no, 4, 4 * fw.scale, d_wodd, o.stream);
  return st;
}

}  // namespace gs

using namespace gs;

// ============================================================================
// C ABI

extern "C" {

const char* gs_strerror(int status) {
  switch (status) {
    case GS_OK: return "success";
    case GS_EINVAL: return "invalid argument";
    case GS_ERANGE: return "value out of the supported range";
    case GS_ENOMEM: return "out of memory or device budget too small";
    case GS_ECUDA: return "CUDA runtime error";
    case GS_ETIMEOUT: return "bounded device wait expired";
    case GS_EUNSUPPORTED: return "weights cannot be summed exactly";
    default: return "unknown status";
  }
}

int gs_num_configs(int npoint, int nb, int64_t* n) {
  if (!n || nb < 1) return GS_EINVAL;
  if (npoint == 3) {
    if (nb > kMaxBins) return GS_ERANGE;
    *n = num_conf3(nb);
    return GS_OK;
  }
  if (npoint == 4) {
    if (nb > kMaxBins4) return GS_ERANGE;
    const int64_t k = nb;
    *n = (k * k * k * k * k * k + 9 * k * k * k * k + 14 * k * k) / 24;
    return GS_OK;
  }
  return GS_EINVAL;
}

int gs_config_bins(int npoint, int nb, int64_t idx, uint8_t* bins, int* chiral) {
  int64_t total = 0;
  int st = gs_num_configs(npoint, nb, &total);
  if (st) return st;
  if (!bins) return GS_EINVAL;
  if (idx < 0 || idx >= total) return GS_ERANGE;
  if (npoint == 3) {
    for (int a = 0; a < nb; ++a)
      for (int b = a; b < nb; ++b)
        for (int c = b; c < nb; ++c)
          if (conf3_rank(a, b, c, nb) == idx) {
            bins[0] = (uint8_t)a;
            bins[1] = (uint8_t)b;
            bins[2] = (uint8_t)c;
            if (chiral) *chiral = 0;
            return GS_OK;
          }
    return GS_ERANGE;
  }
  const Conf4Tables* t = conf4_host(nb, &st);
  if (!t) return st;
  for (int s = 0; s < 6; ++s) bins[s] = t->reps[(size_t)idx * 6 + s];
  if (chiral) *chiral = t->chiral[(size_t)idx];
  return GS_OK;
}

int gs_quantize(const double* pos, int64_t n, int64_t box_u, int periodic, int32_t* xyz,
                const gs_options* options) {
  if ((!pos || !xyz) && n > 0) return GS_EINVAL;
  if (n < 0 || box_u <= 0) return GS_EINVAL;
  if (box_u >= (int64_t(1) << 31)) return GS_ERANGE;
  if (n == 0) return GS_OK;
  const Opts o = read_opts(options);
  int st;
  {
    Scratch sc(o.stream);
    const double* dpos = static_cast<const double*>(to_device(sc, pos, sizeof(double) * 3 * n, o.stream));
    const bool out_dev = is_device_ptr(xyz);
    int32_t* dxyz = out_dev ? xyz : sc.alloc<int32_t>(3 * n);
    if (!dpos || !dxyz) return GS_ENOMEM;
    st = quantize_device(dpos, n, box_u, periodic, dxyz, o.stream, sc);
    if (!st && !out_dev)
      st = cuda_status(cudaMemcpyAsync(xyz, dxyz, sizeof(int32_t) * 3 * n,
                                       cudaMemcpyDeviceToHost, o.stream));
    cudaError_t e = cudaStreamSynchronize(o.stream);
    if (!st) st = cuda_status(e);
  }
  return st;
}

int gs_build_graph(const int32_t* xyz, int64_t n, int64_t box_u, const int64_t* edges_u, int nb,
                   const gs_options* options, gs_graph** out) {
  if (!out || !edges_u || (!xyz && n > 0) || n < 0 || nb < 1 || box_u < 0) return GS_EINVAL;
  *out = nullptr;
  if (nb > kMaxBins || n > kMaxPoints) return GS_ERANGE;
  std::vector<int64_t> edges(edges_u, edges_u + nb + 1);
  if (edges[0] < 0) return GS_ERANGE;
  for (int b = 0; b < nb; ++b)
    if (edges[b + 1] <= edges[b]) return GS_ERANGE;
  if (edges[nb] >= (int64_t(1) << 19)) return GS_ERANGE;
  if (box_u > 0 && (4 * edges[nb] >= box_u || box_u >= (int64_t(1) << 31))) return GS_ERANGE;
  const Opts o = read_opts(options);
  gs_graph* G = new (std::nothrow) gs_graph();
  if (!G) return GS_ENOMEM;
  int st;
  {
    Scratch sc(o.stream);
    const int32_t* dxyz = n ? static_cast<const int32_t*>(
                                  to_device(sc, xyz, sizeof(int32_t) * 3 * n, o.stream))
                            : nullptr;
    if (n && !dxyz) {
      delete G;
      return GS_ENOMEM;
    }
    st = build_graph_device(dxyz, n, box_u, edges, o, &G->g);
    cudaError_t e = cudaStreamSynchronize(o.stream);
    if (!st) st = cuda_status(e);
  }
  if (st) {
    gs_free_graph(G);
    return st;
  }
  *out = G;
  return GS_OK;
}

void gs_free_graph(gs_graph* G) {
  if (!G) return;
  Graph& g = G->g;
  cudaFree(g.d_edges2);
  cudaFree(g.d_xyzp);
  cudaFree(g.d_deg);
  cudaFree(g.d_ptr);
  cudaFree(g.d_adj);
  if (g.h_adj) cudaFreeHost(g.h_adj);
  delete G;
}

int gs_graph_info(const gs_graph* G, gs_graph_stats* s) {
  if (!G || !s) return GS_EINVAL;
  const Graph& g = G->g;
  s->n = g.n;
  s->nb = g.nb;
  s->max_degree = g.max_deg;
  s->edges = g.edges_total;
  s->edge_slots = g.slots;
  s->probe_words = g.probe_words;
  s->bytes_per_edge = sizeof(uint32_t);
  s->device_bytes = g.device_bytes;
  s->windows = g.windows;
  s->cells = g.cells[0];
  if (g.walk_words < 0) {
    const int st = walk_words_device(const_cast<Graph*>(&g));
    if (st) return st;
  }
  s->walk_words = g.walk_words;
  return GS_OK;
}

int gs_graph_tri_words(const gs_graph* G, int64_t* triangles, int64_t* tail_words) {
  if (!G || !triangles || !tail_words) return GS_EINVAL;
  return tri_words_device(G->g, triangles, tail_words);
}

uint64_t gs_kernel_launches(void) { return g_launches.load(); }

namespace gs {
__global__ void k_export_edges(const uint32_t* adj, int64_t slots, int32_t* nbr, uint8_t* bin) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < slots;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t w = adj[i];
    if (nbr) nbr[i] = (w == kSentinel) ? -1 : (int32_t)edge_id(w);
    if (bin) bin[i] = (uint8_t)edge_bin(w);
  }
}
__global__ void k_export_perm(const int4* xyzp, int64_t n, int32_t* perm) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    perm[i] = xyzp[i].w;
}
}  // namespace gs

int gs_graph_export(const gs_graph* G, int64_t* ptr, int32_t* deg, int32_t* nbr, uint8_t* bin,
                    int32_t* perm) {
  if (!G) return GS_EINVAL;
  const Graph& g = G->g;
  cudaStream_t s = nullptr;
  int st = GS_OK;
  {
    Scratch sc(s);
    auto put = [&](void* dst, const void* dsrc, size_t bytes) {
      if (!dst || st) return;
      st = cuda_status(cudaMemcpyAsync(dst, dsrc, bytes, cudaMemcpyDefault, s));
    };
    put(ptr, g.d_ptr, sizeof(int64_t) * (g.n + 1));
    put(deg, g.d_deg, sizeof(int32_t) * g.n);
    if ((nbr || bin) && !st) {
      const uint32_t* adj = g.d_adj;
      if (!adj) {  // out-of-core graph: stage the host copy
        uint32_t* t = sc.alloc<uint32_t>(g.slots);
        if (!t) return GS_ENOMEM;
        st = cuda_status(cudaMemcpyAsync(t, g.h_adj, sizeof(uint32_t) * g.slots,
                                         cudaMemcpyHostToDevice, s));
        adj = t;
      }
      int32_t* dn = nbr ? (is_device_ptr(nbr) ? nbr : sc.alloc<int32_t>(g.slots)) : nullptr;
      uint8_t* db = bin ? (is_device_ptr(bin) ? bin : sc.alloc<uint8_t>(g.slots)) : nullptr;
      if ((nbr && !dn) || (bin && !db)) return GS_ENOMEM;
      if (g.slots) { k_export_edges<<<304, 256, 0, s>>>(adj, g.slots, dn, db); note_launch(); }
      if (nbr && dn != nbr) put(nbr, dn, sizeof(int32_t) * g.slots);
      if (bin && db != bin) put(bin, db, g.slots);
    }
    if (perm && !st) {
      int32_t* dp = is_device_ptr(perm) ? perm : sc.alloc<int32_t>(g.n);
      if (!dp) return GS_ENOMEM;
      if (g.n) { k_export_perm<<<304, 256, 0, s>>>(g.d_xyzp, g.n, dp); note_launch(); }
      if (dp != perm) put(perm, dp, sizeof(int32_t) * g.n);
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (!st) st = cuda_status(e);
  }
  return st;
}

// Runs a counting call: device staging of outputs, weights, the launcher and
// the copy back of results.
namespace gs {
struct OutBuf {
  void* user;
  void* dev;
  size_t bytes;
};
}  // namespace gs

int gs_count_3pcf(const gs_graph* G, const float* w, uint64_t* counts, double* wsum,
                  const gs_options* options) {
  if (!G || !counts) return GS_EINVAL;
  const Graph& g = G->g;
  const Opts o = read_opts(options);
  const int64_t nc = num_conf3(g.nb);
  int st = GS_OK;
  {
    Scratch sc(o.stream);
    FixedW fw;
    if (w) {
      st = prepare_weights(g, w, &fw, sc, o.stream, 54);
      if (st) return st;
    }
    uint64_t* dc = is_device_ptr(counts) ? counts : sc.alloc<uint64_t>(nc);
    double* dw = wsum ? (is_device_ptr(wsum) ? wsum : sc.alloc<double>(nc)) : nullptr;
    if (!dc || (wsum && !dw)) return GS_ENOMEM;
    if (w && wsum && fw.bits > kNarrowWeightBits)
      st = count3_wide(g, fw, dc, dw, o, sc);
    else
      st = count3_device(g, w ? &fw : nullptr, dc, dw, o, sc);
    if (!st && dc != counts)
      st = cuda_status(cudaMemcpyAsync(counts, dc, sizeof(uint64_t) * nc, cudaMemcpyDeviceToHost, o.stream));
    if (!st && dw && dw != wsum)
      st = cuda_status(cudaMemcpyAsync(wsum, dw, sizeof(double) * nc, cudaMemcpyDeviceToHost, o.stream));
    cudaError_t e = cudaStreamSynchronize(o.stream);
    if (!st) st = cuda_status(e);
  }
  return st;
}

int gs_count_3pcf_batch(const gs_graph* const* graphs, int32_t n_graphs, const float* const* w,
                        uint64_t* const* counts, double* const* wsum, const gs_options* options) {
  if (!graphs || !counts || n_graphs < 1) return GS_EINVAL;
  const int nb = graphs[0] ? graphs[0]->g.nb : 0;
  for (int k = 0; k < n_graphs; ++k) {
    if (!graphs[k] || !counts[k] || graphs[k]->g.nb != nb) return GS_EINVAL;
    if (!graphs[k]->g.d_adj) return GS_EINVAL;  // out-of-core graphs are counted one by one
    if (w && !w[k]) return GS_EINVAL;
  }
  const Opts o = read_opts(options);
  const int64_t nc = num_conf3(nb);
  int st = GS_OK;
  {
    Scratch sc(o.stream);
    std::vector<FixedW> fws(w ? n_graphs : 0);
    std::vector<const Graph*> gr(n_graphs);
    std::vector<uint64_t*> dc(n_graphs);
    std::vector<double*> dw(wsum ? n_graphs : 0);
    for (int k = 0; k < n_graphs; ++k) {
      gr[k] = &graphs[k]->g;
      if (w) {
        st = prepare_weights(*gr[k], w[k], &fws[k], sc, o.stream);
        if (st) return st;
      }
      dc[k] = is_device_ptr(counts[k]) ? counts[k] : sc.alloc<uint64_t>(nc);
      if (!dc[k]) return GS_ENOMEM;
      if (wsum) {
        dw[k] = !wsum[k] ? nullptr : (is_device_ptr(wsum[k]) ? wsum[k] : sc.alloc<double>(nc));
        if (wsum[k] && !dw[k]) return GS_ENOMEM;
      }
    }
    st = count3_batch_device(gr.data(), n_graphs, w ? fws.data() : nullptr, dc.data(),
                             wsum ? dw.data() : nullptr, o, sc);
    for (int k = 0; k < n_graphs && !st; ++k) {
      if (dc[k] != counts[k])
        st = cuda_status(cudaMemcpyAsync(counts[k], dc[k], sizeof(uint64_t) * nc, cudaMemcpyDeviceToHost, o.stream));
      if (!st && wsum && wsum[k] && dw[k] != wsum[k])
        st = cuda_status(cudaMemcpyAsync(wsum[k], dw[k], sizeof(double) * nc, cudaMemcpyDeviceToHost, o.stream));
    }
    cudaError_t e = cudaStreamSynchronize(o.stream);
    if (!st) st = cuda_status(e);
  }
  return st;
}

static int count4_common(const gs_graph* G, const float* w, bool parity, uint64_t* even,
                         int64_t* odd, double* weven, double* wodd, const gs_options* options,
                         bool pix = false) {
  if (!G || !even) return GS_EINVAL;
  const Graph& g = G->g;
  const Opts o = read_opts(options);
  int st = GS_OK;
  const Conf4Tables* t = conf4_tables(g.nb, &st);
  if (!t) return st;
  const int64_t nc = t->n_orbits;
  {
    Scratch sc(o.stream);
    FixedW fw;
    if (w) {
      st = prepare_weights(g, w, &fw, sc, o.stream, 52);
      if (st) return st;
    }
    uint64_t* de = is_device_ptr(even) ? even : sc.alloc<uint64_t>(nc);
    int64_t* dod = odd ? (is_device_ptr(odd) ? odd : sc.alloc<int64_t>(nc)) : nullptr;
    double* dwe = weven ? (is_device_ptr(weven) ? weven : sc.alloc<double>(nc)) : nullptr;
    double* dwo = wodd ? (is_device_ptr(wodd) ? wodd : sc.alloc<double>(nc)) : nullptr;
    if (!de || (odd && !dod) || (weven && !dwe) || (wodd && !dwo)) return GS_ENOMEM;
    if (w && fw.bits > kNarrowWeightBits)
      st = count4_wide(g, fw, parity, pix, de, dod, dwe, dwo, o, sc);
    else
      st = count4_device(g, w ? &fw : nullptr, parity, de, dod, dwe, dwo, o, sc, pix);
    OutBuf outs[4] = {{even, de, sizeof(uint64_t) * nc},
                      {odd, dod, sizeof(int64_t) * nc},
                      {weven, dwe, sizeof(double) * nc},
                      {wodd, dwo, sizeof(double) * nc}};
    for (auto& b : outs)
      if (!st && b.user && b.dev != b.user)
        st = cuda_status(cudaMemcpyAsync(b.user, b.dev, b.bytes, cudaMemcpyDeviceToHost, o.stream));
    cudaError_t e = cudaStreamSynchronize(o.stream);
    if (!st) st = cuda_status(e);
  }
  return st;
}

int gs_count_4pcf(const gs_graph* G, const float* w, uint64_t* counts, double* wsum,
                  const gs_options* options) {
  return count4_common(G, w, false, counts, nullptr, wsum, nullptr, options);
}

int gs_count_4pcf_parity(const gs_graph* G, const float* w, uint64_t* even, int64_t* odd,
                         double* weven, double* wodd, const gs_options* options) {
  if (!odd) return GS_EINVAL;
  return count4_common(G, w, true, even, odd, weven, wodd, options);
}

int gs_count_4pcf_parity_pix(const gs_graph* G, const float* w, uint64_t* even, int64_t* odd,
                             double* weven, double* wodd, const gs_options* options) {
  if (!odd) return GS_EINVAL;
  return count4_common(G, w, true, even, odd, weven, wodd, options, true);
}

int gs_direction_pixels(const int32_t* dirs, int64_t n, uint8_t* pixels,
                        const gs_options* options) {
  if (n < 0 || (n > 0 && (!dirs || !pixels))) return GS_EINVAL;
  const Opts o = read_opts(options);
  int st = GS_OK;
  {
    Scratch sc(o.stream);
    const int32_t* dd = static_cast<const int32_t*>(to_device(sc, dirs, sizeof(int32_t) * 3 * n, o.stream));
    uint8_t* dp = is_device_ptr(pixels) ? pixels : sc.alloc<uint8_t>(n > 0 ? n : 1);
    if (n > 0 && (!dd || !dp)) return GS_ENOMEM;
    st = direction_pixels_device(dd, n, dp, o.stream);
    if (!st && n > 0 && dp != pixels)
      st = cuda_status(cudaMemcpyAsync(pixels, dp, (size_t)n, cudaMemcpyDeviceToHost, o.stream));
    cudaError_t e = cudaStreamSynchronize(o.stream);
    if (!st) st = cuda_status(e);
  }
  return st;
}

int gs_disconnected_4pcf(const gs_graph* G, const float* w, const double* rr, uint64_t* pairs,
                         double* xi, double* zeta_disc, const gs_options* options) {
  if (!G) return GS_EINVAL;
  const Graph& g = G->g;
  if (!rr && g.box_u == 0) return GS_EINVAL;
  const Opts o = read_opts(options);
  int st = GS_OK;
  int64_t no = 0;
  if (zeta_disc) {
    st = gs_num_configs(4, g.nb, &no);
    if (st) return st;
  }
  {
    Scratch sc(o.stream);
    FixedW fw;
    if (w) {
      st = prepare_weights(g, w, &fw, sc, o.stream);
      if (st) return st;
    }
    const double* drr = static_cast<const double*>(to_device(sc, rr, sizeof(double) * g.nb, o.stream));
    uint64_t* dp = pairs ? (is_device_ptr(pairs) ? pairs : sc.alloc<uint64_t>(g.nb)) : nullptr;
    double* dx = xi ? (is_device_ptr(xi) ? xi : sc.alloc<double>(g.nb)) : nullptr;
    double* dz = zeta_disc ? (is_device_ptr(zeta_disc) ? zeta_disc : sc.alloc<double>(no)) : nullptr;
    if ((rr && !drr) || (pairs && !dp) || (xi && !dx) || (zeta_disc && !dz)) return GS_ENOMEM;
    st = pairs_disc_device(g, w ? &fw : nullptr, drr, dp, dx, dz, o, sc);
    OutBuf outs[3] = {{pairs, dp, sizeof(uint64_t) * g.nb},
                      {xi, dx, sizeof(double) * g.nb},
                      {zeta_disc, dz, sizeof(double) * no}};
    for (auto& b : outs)
      if (!st && b.user && b.dev != b.user)
        st = cuda_status(cudaMemcpyAsync(b.user, b.dev, b.bytes, cudaMemcpyDeviceToHost, o.stream));
    cudaError_t e = cudaStreamSynchronize(o.stream);
    if (!st) st = cuda_status(e);
  }
  return st;
}

int gs_count_3pcf_equilateral(const gs_graph* G, const float* w, uint64_t* counts, double* wsum,
                              const gs_options* options) {
  if (!G || !counts || (wsum && !w)) return GS_EINVAL;
  const Graph& g = G->g;
  const Opts o = read_opts(options);
  int st = GS_OK;
  {
    Scratch sc(o.stream);
    FixedW fw;
    if (w) {
      st = prepare_weights(g, w, &fw, sc, o.stream);
      if (st) return st;
    }
    uint64_t* dc = is_device_ptr(counts) ? counts : sc.alloc<uint64_t>(g.nb);
    double* dw = wsum ? (is_device_ptr(wsum) ? wsum : sc.alloc<double>(g.nb)) : nullptr;
    if (!dc || (wsum && !dw)) return GS_ENOMEM;
    st = count3_device(g, w ? &fw : nullptr, dc, dw, o, sc, /*equi=*/true);
    OutBuf outs[2] = {{counts, dc, sizeof(uint64_t) * g.nb}, {wsum, dw, sizeof(double) * g.nb}};
    for (auto& b : outs)
      if (!st && b.user && b.dev != b.user)
        st = cuda_status(cudaMemcpyAsync(b.user, b.dev, b.bytes, cudaMemcpyDeviceToHost, o.stream));
    cudaError_t e = cudaStreamSynchronize(o.stream);
    if (!st) st = cuda_status(e);
  }
  return st;
}

int gs_count_3pcf_mu(const gs_graph* G, const float* w, int32_t nmu, uint64_t* counts,
                     double* wsum, const gs_options* options) {
  if (!G || !counts || (wsum && !w) || nmu < 1 || nmu > 64) return GS_EINVAL;
  const Graph& g = G->g;
  const Opts o = read_opts(options);
  const int64_t ncell = num_conf3(g.nb) * (nmu + 1);
  int st = GS_OK;
  {
    Scratch sc(o.stream);
    FixedW fw;
    if (w) {
      st = prepare_weights(g, w, &fw, sc, o.stream);
      if (st) return st;
    }
    uint64_t* dc = is_device_ptr(counts) ? counts : sc.alloc<uint64_t>(ncell);
    double* dw = wsum ? (is_device_ptr(wsum) ? wsum : sc.alloc<double>(ncell)) : nullptr;
    if (!dc || (wsum && !dw)) return GS_ENOMEM;
    st = count3mu_device(g, w ? &fw : nullptr, nmu, dc, dw, o, sc);
    OutBuf outs[2] = {{counts, dc, sizeof(uint64_t) * ncell}, {wsum, dw, sizeof(double) * ncell}};
    for (auto& b : outs)
      if (!st && b.user && b.dev != b.user)
        st = cuda_status(cudaMemcpyAsync(b.user, b.dev, b.bytes, cudaMemcpyDeviceToHost, o.stream));
    cudaError_t e = cudaStreamSynchronize(o.stream);
    if (!st) st = cuda_status(e);
  }
  return st;
}

int gs_connected_4pcf(const gs_graph* G_dr, const float* w_signed, const gs_graph* G_r,
                      const float* w_r, double* xi, double* zeta_even, double* zeta_odd,
                      double* zeta_disc, double* zeta_conn, const gs_options* options) {
  if (!G_dr || !G_r || !w_signed || !w_r) return GS_EINVAL;
  const Graph& gdr = G_dr->g;
  const Graph& gr = G_r->g;
  if (gdr.nb != gr.nb) return GS_EINVAL;
  if (gdr.edges != gr.edges) return GS_EINVAL;  // both graphs on the same bins
  const Opts o = read_opts(options);
  if (o.shards > 1) return GS_EINVAL;  // the ratios do not add over hub shards
  int64_t no = 0;
  int st = gs_num_configs(4, gdr.nb, &no);
  if (st) return st;
  {
    Scratch sc(o.stream);
    FixedW fdr, fr;
    st = prepare_weights(gdr, w_signed, &fdr, sc, o.stream);
    if (!st) st = prepare_weights(gr, w_r, &fr, sc, o.stream);
    if (st) return st;
    auto dev_out = [&](double* p, int64_t n) -> double* {
      return !p ? nullptr : (is_device_ptr(p) ? p : sc.alloc<double>(n));
    };
    double* dx = dev_out(xi, gdr.nb);
    double* de = dev_out(zeta_even, no);
    double* dod = dev_out(zeta_odd, no);
    double* dd = dev_out(zeta_disc, no);
    double* dc = dev_out(zeta_conn, no);
    if ((xi && !dx) || (zeta_even && !de) || (zeta_odd && !dod) || (zeta_disc && !dd) ||
        (zeta_conn && !dc))
      return GS_ENOMEM;
    st = connected_device(gdr, fdr, gr, fr, dx, de, dod, dd, dc, o, sc);
    OutBuf outs[5] = {{xi, dx, sizeof(double) * gdr.nb},
                      {zeta_even, de, sizeof(double) * no},
                      {zeta_odd, dod, sizeof(double) * no},
                      {zeta_disc, dd, sizeof(double) * no},
                      {zeta_conn, dc, sizeof(double) * no}};
    for (auto& b : outs)
      if (!st && b.user && b.dev != b.user)
        st = cuda_status(cudaMemcpyAsync(b.user, b.dev, b.bytes, cudaMemcpyDeviceToHost, o.stream));
    cudaError_t e = cudaStreamSynchronize(o.stream);
    if (!st) st = cuda_status(e);
  }
  return st;
}

}  // extern "C"
