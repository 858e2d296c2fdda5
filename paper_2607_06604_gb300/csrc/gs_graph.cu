// Lattice quantisation and the device radius-search graph build (Sec. 2.1).
//
// Points are binned into a uniform cell grid whose cells are at least
// E_nb wide, so every neighbour lies in the 27 surrounding cells. Points are
// relabelled in cell order (cell-major, caller index within a cell), which
// makes rows come out sorted when the stencil cells are visited in
// increasing cell order, and keeps neighbour ids close to the hub id (good
// L2 locality for the counting kernels). Only the oriented half
// N+(i) = {j > i} is stored: every tuple is counted at its smallest label.
#include <algorithm>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kMaxCellsPerAxis = 256;
constexpr int kCellThreads = 512;   // row pass: one CTA per cell
constexpr int kCellCap = 4096;      // stencil points staged in shared memory (64 KB)

struct GridDesc {
  int nc[3];
  int64_t lo[3];     // open box: grid origin
  int64_t width[3];  // open box: cell width
  int64_t box;       // periodic box side, 0 = open
};

__device__ inline int cell_axis(const GridDesc& G, int a, int x) {
  if (G.box) return (int)(((int64_t)x * G.nc[a]) / G.box);
  return (int)(((int64_t)x - G.lo[a]) / G.width[a]);
}

__device__ inline int64_t min_image(int64_t d, int64_t box) {
  if (box) {
    if (2 * d >= box) d -= box;
    else if (2 * d < -box) d += box;
  }
  return d;
}

__global__ void k_quantize(const double* pos, int64_t n3, int64_t box_u, int periodic,
                           int32_t* out, int* err) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n3;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double s = pos[i] * 1024.0;  // exact: scaling by a power of two
    double f = floor(s);
    if (!(f > -9.0e15 && f < 9.0e15)) {  // not finite or beyond exact integers
      atomicOr(err, kErrRange);
      out[i] = 0;
      continue;
    }
    int64_t X = (int64_t)f;
    if (periodic) {
      X %= box_u;
      if (X < 0) X += box_u;
    } else if (X < 0 || X >= box_u) {
      atomicOr(err, kErrRange);
      X = 0;
    }
    out[i] = (int32_t)X;
  }
}

// Validates coordinates and computes the bounding box.
__global__ void k_check_bbox(const int32_t* xyz, int64_t n, int64_t box, int* bbox, int* err) {
  int mn[3] = {INT_MAX, INT_MAX, INT_MAX}, mx[3] = {INT_MIN, INT_MIN, INT_MIN};
  int bad = 0;
  const int64_t limit = box ? box : (int64_t(1) << 30);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    for (int a = 0; a < 3; ++a) {
      const int x = xyz[3 * i + a];
      if (x < 0 || (int64_t)x >= limit) bad = 1;
      mn[a] = min(mn[a], x);
      mx[a] = max(mx[a], x);
    }
  }
  for (int o = 16; o; o >>= 1) {
    for (int a = 0; a < 3; ++a) {
      mn[a] = min(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], o));
      mx[a] = max(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], o));
    }
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    for (int a = 0; a < 3; ++a) {
      atomicMin(bbox + a, mn[a]);
      atomicMax(bbox + 3 + a, mx[a]);
    }
    if (bad) atomicOr(err, kErrRange);
  }
}

__global__ void k_cell_keys(const int32_t* xyz, int64_t n, GridDesc G, int32_t* key,
                            int32_t* count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int cx = cell_axis(G, 0, xyz[3 * i]);
    const int cy = cell_axis(G, 1, xyz[3 * i + 1]);
    const int cz = cell_axis(G, 2, xyz[3 * i + 2]);
    const int c = (cx * G.nc[1] + cy) * G.nc[2] + cz;
    key[i] = c;
    atomicAdd(count + c, 1);
  }
}

// Groups points by cell (order inside a cell is arbitrary here).
__global__ void k_scatter(const int32_t* key, int64_t n, int32_t* cursor, int32_t* tmp) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int pos = atomicAdd(cursor + key[i], 1);
    tmp[pos] = (int32_t)i;
  }
}

// Orders each cell by caller index: slot s goes to cell_start + rank, rank =
// number of points of the same cell with a smaller caller index.
__global__ void k_rank_in_cell(const int32_t* key, const int32_t* tmp, int64_t n,
                               const int32_t* cell_start, const int32_t* cell_count,
                               const int32_t* xyz, int4* xyzp) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n;
       s += (int64_t)gridDim.x * blockDim.x) {
    const int32_t me = tmp[s];
    const int c = key[me];
    const int b = cell_start[c], e = b + cell_count[c];
    int r = 0;
    for (int t = b; t < e; ++t) r += tmp[t] < me;
    xyzp[b + r] = make_int4(xyz[3 * (int64_t)me], xyz[3 * (int64_t)me + 1],
                            xyz[3 * (int64_t)me + 2], me);
  }
}

// Warp-wide ascending sort of one int per lane (bitonic network).
__device__ inline int warp_sort_asc(int v) {
  const int lane = threadIdx.x & 31;
  for (int k = 2; k <= 32; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      const int o = __shfl_xor_sync(0xffffffffu, v, j);
      const bool up = ((lane & k) == 0);
      const bool lower = ((lane & j) == 0);
      const int mn = min(v, o), mx = max(v, o);
      v = (lower == up) ? mn : mx;
    }
  return v;
}

// Squared minimum-image distance of a candidate pair, or a value >= E_nb^2
// when the pair cannot be an edge. SMALL: E_nb <= 2^16 and every
// coordinate difference fits 31 bits (box or extent below 2^30), so the
// test runs in 32-bit arithmetic: a pair with any |component| >= 2^16 is no
// edge, and otherwise each squared component is below 2^32.
template <bool SMALL>
__device__ inline int64_t cand_d2(const int4& P, const int4& Q, int64_t box, int64_t e2hi) {
  if constexpr (SMALL) {
    const int bx = (int)box;
    auto mi32 = [bx](int d) {
      if (bx) {
        if (2 * d >= bx) d -= bx;
        else if (2 * d < -bx) d += bx;
      }
      return d;
    };
    const unsigned ax = (unsigned)abs(mi32(Q.x - P.x)), ay = (unsigned)abs(mi32(Q.y - P.y)),
                   az = (unsigned)abs(mi32(Q.z - P.z));
    return (max(ax, max(ay, az)) >= 65536u)
               ? e2hi
               : (int64_t)((unsigned long long)(ax * ax) + (ay * ay) + (az * az));
  } else {
    const int64_t dx = min_image((int64_t)Q.x - P.x, box);
    const int64_t dy = min_image((int64_t)Q.y - P.y, box);
    const int64_t dz = min_image((int64_t)Q.z - P.z, box);
    return dx * dx + dy * dy + dz * dz;
  }
}

// Row pass, one CTA per cell (persistent over cells): every hub of a cell
// has the same stencil, the cells with index >= its own (in increasing
// order, so rows come out sorted). The CTA copies the points of those
// cells into shared memory once (up to cap points; a cell whose stencil
// holds more reads them from global memory), then each warp takes one hub
// of the cell at a time and tests every candidate j > i.
// FILL = false counts |N+(i)|; FILL = true writes the packed words. Only
// hubs in [h0, h1) are processed (chunked out-of-core builds).
template <bool FILL, bool SMALL>
__global__ void __launch_bounds__(kCellThreads) k_rows_cells(
    const int4* __restrict__ xyzp, GridDesc G, int64_t ncell, const int32_t* __restrict__ cell_start,
    const int32_t* __restrict__ cell_count, const int64_t* __restrict__ e2g, int nb,
    int32_t* deg, const int64_t* __restrict__ ptr, uint32_t* __restrict__ adj, int64_t h0,
    int64_t h1, int64_t out_off, int cap) {
  extern __shared__ int4 s_cand[];
  __shared__ int64_t e2[kMaxBins + 1];
  __shared__ int s_beg[27], s_cnt[27], s_off[28], s_cell[27];
  __shared__ int s_ncell;
  for (int b = threadIdx.x; b <= nb; b += blockDim.x) e2[b] = e2g[b];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int kW = kCellThreads / 32;
  const int64_t e2lo = e2[0], e2hi = e2[nb];
  for (int64_t own = blockIdx.x; own < ncell; own += gridDim.x) {
    const int64_t cb = cell_start[own], ce = cb + cell_count[own];
    const int64_t hb = cb > h0 ? cb : h0, he = ce < h1 ? ce : h1;
    if (hb >= he) continue;  // the same decision in every thread
    if (warp == 0) {
      const int c2 = (int)(own % G.nc[2]), c1 = (int)((own / G.nc[2]) % G.nc[1]),
                c0 = (int)(own / ((int64_t)G.nc[1] * G.nc[2]));
      int cell = INT_MAX;
      if (lane < 27) {
        int q[3] = {c0 + lane / 9 - 1, c1 + (lane / 3) % 3 - 1, c2 + lane % 3 - 1};
        bool ok = true;
        for (int a = 0; a < 3; ++a) {
          if (G.box) q[a] = (q[a] + G.nc[a]) % G.nc[a];
          else if (q[a] < 0 || q[a] >= G.nc[a]) ok = false;
        }
        if (ok) cell = (q[0] * G.nc[1] + q[1]) * G.nc[2] + q[2];
        if (cell < own) cell = INT_MAX;
      }
      cell = warp_sort_asc(cell);
      const int prev = __shfl_up_sync(0xffffffffu, cell, 1);
      if (lane > 0 && prev == cell) cell = INT_MAX;  // duplicate stencil cell
      cell = warp_sort_asc(cell);                    // valid cells first
      const unsigned valid = __ballot_sync(0xffffffffu, cell != INT_MAX);
      int c = 0;
      if (cell != INT_MAX) {
        s_cell[lane] = cell;
        s_beg[lane] = cell_start[cell];
        c = cell_count[cell];
        s_cnt[lane] = c;
      }
      // exclusive offsets of the cells' points in the staged copy
      int incl = c;
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      if (lane < 27) s_off[lane + 1] = incl;
      if (lane == 0) {
        s_off[0] = 0;
        s_ncell = __popc(valid);
      }
    }
    __syncthreads();
    const int ncs = s_ncell;
    const bool staged = s_off[ncs] <= cap;
    if (staged) {
      for (int k = 0; k < ncs; ++k)
        for (int t = threadIdx.x; t < s_cnt[k]; t += kCellThreads)
          s_cand[s_off[k] + t] = xyzp[(int64_t)s_beg[k] + t];
    }
    __syncthreads();
    for (int64_t i = hb + warp; i < he; i += kW) {
      const int4 P = xyzp[i];
      int64_t count = 0;
      int64_t out = FILL ? ptr[i] - out_off : 0;
      for (int k = 0; k < ncs; ++k) {
        const int64_t b = s_beg[k], e = b + s_cnt[k];
        const int64_t st = (s_cell[k] == own) ? i + 1 : b;
        const int sk = s_off[k];
        for (int64_t t0 = st; t0 < e; t0 += 32) {
          const int64_t t = t0 + lane;
          bool hit = false;
          uint32_t word = 0;
          if (t < e) {
            const int4 Q = staged ? s_cand[sk + (int)(t - b)] : xyzp[t];
            const int64_t D2 = cand_d2<SMALL>(P, Q, G.box, e2hi);
            if (D2 >= e2lo && D2 < e2hi) {
              hit = true;
              if (FILL) {
                int lo = 0, hi = nb;
                while (hi - lo > 1) {
                  const int mid = (lo + hi) >> 1;
                  if (e2[mid] <= D2) lo = mid;
                  else hi = mid;
                }
                word = ((uint32_t)t << 8) | (uint32_t)lo;
              }
            }
          }
          const unsigned m = __ballot_sync(0xffffffffu, hit);
          if (FILL && hit) adj[out + __popc(m & ((1u << lane) - 1u))] = word;
          out += __popc(m);
          count += __popc(m);
        }
      }
      if (!FILL) {
        if (lane == 0) deg[i] = (int32_t)count;
      } else {
        const int64_t end = ptr[i + 1] - out_off;
        for (int64_t p = out + lane; p < end; p += 32) adj[p] = kSentinel;
      }
    }
    __syncthreads();  // the staged copy is rewritten for the next cell
  }
}

__global__ void k_pad_lengths(const int32_t* deg, int64_t n, int64_t* len) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n;
       i += (int64_t)gridDim.x * blockDim.x)
    len[i] = (i < n) ? pad_row(deg[i]) : 0;
}

// probe[i] = sum over j in N+(i) of |N+(j)|, and the largest degree.
__global__ void k_graph_stats(const int32_t* __restrict__ deg, const int64_t* __restrict__ ptr,
                              const uint32_t* __restrict__ adj, int64_t adj_off, int64_t h0,
                              int64_t h1, unsigned long long* probe_total,
                              unsigned long long* edge_total, int* max_deg) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  unsigned long long pw = 0, ew = 0;
  int md = 0;
  for (int64_t i = h0 + blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < h1;
       i += warps) {
    const int d = deg[i];
    const int64_t p = ptr[i] - adj_off;
    for (int k = lane; k < d; k += 32) pw += (unsigned long long)deg[edge_id(adj[p + k])];
    if (lane == 0) {
      ew += (unsigned long long)d;
      md = max(md, d);
    }
  }
  for (int o = 16; o; o >>= 1) {
    pw += __shfl_xor_sync(0xffffffffu, pw, o);
    ew += __shfl_xor_sync(0xffffffffu, ew, o);
    md = max(md, __shfl_xor_sync(0xffffffffu, md, o));
  }
  if (lane == 0) {
    atomicAdd(probe_total, pw);
    atomicAdd(edge_total, ew);
    atomicMax(max_deg, md);
  }
}

int grid_blocks(int64_t work, int threads) {
  int64_t b = (work + threads - 1) / threads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 16));
}

}  // namespace

int quantize_device(const double* d_pos, int64_t n, int64_t box_u, int periodic, int32_t* d_xyz,
                    cudaStream_t s, Scratch& sc) {
  int* err = sc.alloc<int>(1);
  if (!err) return GS_ENOMEM;
  cudaMemsetAsync(err, 0, sizeof(int), s);
  { k_quantize<<<grid_blocks(3 * n, 256), 256, 0, s>>>(d_pos, 3 * n, box_u, periodic, d_xyz, err); note_launch(); }
  int h = 0;
  cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e);
  return h ? GS_ERANGE : GS_OK;
}

int build_graph_device(const int32_t* d_xyz, int64_t n, int64_t box_u,
                       const std::vector<int64_t>& edges, const Opts& o, Graph* g) {
  cudaStream_t s = o.stream;
  cudaGetDevice(&g->device);
  g->n = n;
  g->nb = (int)edges.size() - 1;
  g->box_u = box_u;
  g->budget = o.budget;
  g->force_windows = std::max(0, o.force_windows);
  g->edges = edges;
  const int nb = g->nb;
  const int64_t rmax = edges[nb];
  std::vector<int64_t> e2(nb + 1);
  for (int b = 0; b <= nb; ++b) e2[b] = edges[b] * edges[b];
  auto dev_alloc = [&](void** p, size_t bytes) -> int {
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return GS_ENOMEM;
    }
    g->device_bytes += (int64_t)bytes;
    return GS_OK;
  };
  int st = dev_alloc((void**)&g->d_edges2, sizeof(int64_t) * (nb + 1));
  if (!st) st = dev_alloc((void**)&g->d_xyzp, sizeof(int4) * std::max<int64_t>(n, 1));
  if (!st) st = dev_alloc((void**)&g->d_deg, sizeof(int32_t) * std::max<int64_t>(n, 1));
  if (!st) st = dev_alloc((void**)&g->d_ptr, sizeof(int64_t) * (n + 1));
  if (st) return st;
  cudaMemcpyAsync(g->d_edges2, e2.data(), sizeof(int64_t) * (nb + 1), cudaMemcpyHostToDevice, s);
  if (n == 0) {
    cudaMemsetAsync(g->d_ptr, 0, sizeof(int64_t), s);
    g->h_ptr.assign(1, 0);
    return dev_alloc((void**)&g->d_adj, 16);
  }

  Scratch sc(s);
  int* flags = sc.alloc<int>(8);  // bbox min[3], max[3], err
  if (!flags) return GS_ENOMEM;
  const int init[8] = {INT_MAX, INT_MAX, INT_MAX, INT_MIN, INT_MIN, INT_MIN, 0, 0};
  cudaMemcpyAsync(flags, init, sizeof(init), cudaMemcpyHostToDevice, s);
  { k_check_bbox<<<grid_blocks(n, 256), 256, 0, s>>>(d_xyz, n, box_u, flags, flags + 6); note_launch(); }
  int h[8];
  cudaMemcpyAsync(h, flags, sizeof(h), cudaMemcpyDeviceToHost, s);
  cudaError_t ce = cudaStreamSynchronize(s);
  if (ce != cudaSuccess) return cuda_status(ce);
  if (h[6]) return GS_ERANGE;

  GridDesc G;
  G.box = box_u;
  for (int a = 0; a < 3; ++a) {
    if (box_u) {
      G.nc[a] = (int)std::max<int64_t>(1, std::min<int64_t>(box_u / rmax, kMaxCellsPerAxis));
      G.lo[a] = 0;
      G.width[a] = 0;
    } else {
      const int64_t ext = (int64_t)h[3 + a] - h[a];
      G.lo[a] = h[a];
      G.width[a] = std::max<int64_t>(rmax, ext / kMaxCellsPerAxis + 1);
      G.nc[a] = (int)(ext / G.width[a] + 1);
    }
    g->cells[a] = G.nc[a];
  }
  const int64_t ncell = (int64_t)G.nc[0] * G.nc[1] * G.nc[2];

  int32_t* key = sc.alloc<int32_t>(n);
  int32_t* tmp = sc.alloc<int32_t>(n);
  int32_t* cnt = sc.alloc<int32_t>(ncell);
  int32_t* start = sc.alloc<int32_t>(ncell);
  int32_t* cursor = sc.alloc<int32_t>(ncell);
  int64_t* len = sc.alloc<int64_t>(n + 1);
  if (!key || !tmp || !cnt || !start || !cursor || !len) return GS_ENOMEM;
  cudaMemsetAsync(cnt, 0, sizeof(int32_t) * ncell, s);
  { k_cell_keys<<<grid_blocks(n, 256), 256, 0, s>>>(d_xyz, n, G, key, cnt); note_launch(); }
  st = scan_exclusive_i32(cnt, start, ncell, nullptr, s, sc);
  if (st) return st;
  cudaMemcpyAsync(cursor, start, sizeof(int32_t) * ncell, cudaMemcpyDeviceToDevice, s);
  { k_scatter<<<grid_blocks(n, 256), 256, 0, s>>>(key, n, cursor, tmp); note_launch(); }
  { k_rank_in_cell<<<grid_blocks(n, 256), 256, 0, s>>>(key, tmp, n, start, cnt, d_xyz, g->d_xyzp); note_launch(); }

  // row passes: persistent CTAs over the cells
  const size_t cell_smem = (size_t)kCellCap * sizeof(int4);
  // 32-bit candidate tests when E_nb <= 2^16 and coordinate differences fit
  // 31 bits
  // (variant bit 1: the 64-bit test everywhere)
  bool small = rmax <= 65536 && !(o.variant & 1);
  for (int a = 0; a < 3 && small; ++a)
    small = box_u ? box_u < (int64_t(1) << 30) : (int64_t)h[3 + a] - h[a] < (int64_t(1) << 30);
  auto rows_count = small ? k_rows_cells<false, true> : k_rows_cells<false, false>;
  auto rows_fill = small ? k_rows_cells<true, true> : k_rows_cells<true, false>;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  for (auto k : {rows_count, rows_fill})
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cell_smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rows_fill, kCellThreads, cell_smem);
  const int row_blocks = (int)std::min<int64_t>(ncell, (int64_t)std::max(1, per_sm) * sms * 8);
  KernelTimer timer(o.kernel_ms);
  timer.start(s);
  { rows_count<<<row_blocks, kCellThreads, cell_smem, s>>>(g->d_xyzp, G, ncell, start, cnt,
                                                          g->d_edges2, nb, g->d_deg, nullptr,
                                                          nullptr, 0, n, 0, kCellCap); note_launch(); }
  timer.stop(s);
  { k_pad_lengths<<<grid_blocks(n + 1, 256), 256, 0, s>>>(g->d_deg, n, len); note_launch(); }
  st = scan_exclusive_i64(len, g->d_ptr, n + 1, s, sc);
  if (st) return st;
  g->h_ptr.resize(n + 1);
  cudaMemcpyAsync(g->h_ptr.data(), g->d_ptr, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, s);
  ce = cudaStreamSynchronize(s);
  if (ce != cudaSuccess) return cuda_status(ce);
  g->slots = g->h_ptr[n];
  unsigned long long* tot = sc.alloc<unsigned long long>(3);
  if (!tot) return GS_ENOMEM;
  cudaMemsetAsync(tot, 0, sizeof(unsigned long long) * 3, s);
  const uint64_t edge_bytes = sizeof(uint32_t) * (uint64_t)g->slots;
  const bool out_of_core = o.force_windows > 0 || (o.budget && edge_bytes > o.budget);
  if (!out_of_core) {
    st = dev_alloc((void**)&g->d_adj, edge_bytes);
    if (st) return st;
    timer.start(s);
    { rows_fill<<<row_blocks, kCellThreads, cell_smem, s>>>(g->d_xyzp, G, ncell, start, cnt,
                                                           g->d_edges2, nb, g->d_deg, g->d_ptr,
                                                           g->d_adj, 0, n, 0, kCellCap); note_launch(); }
    timer.stop(s);
    { k_graph_stats<<<grid_blocks(n * 32, 256), 256, 0, s>>>(g->d_deg, g->d_ptr, g->d_adj, 0, 0, n, tot,
                                                           tot + 1, (int*)(tot + 2)); note_launch(); }
  } else {
    // Out of core: the edges live in pinned host memory. Rows are filled a
    // chunk of hubs at a time into a device staging buffer and copied out.
    ce = cudaHostAlloc((void**)&g->h_adj, std::max<uint64_t>(edge_bytes, 16), cudaHostAllocDefault);
    if (ce != cudaSuccess) {
      cudaGetLastError();
      g->h_adj = nullptr;
      return GS_ENOMEM;
    }
    int64_t chunk = o.budget ? (int64_t)(o.budget / (2 * sizeof(uint32_t))) : g->slots;
    if (o.force_windows > 0)
      chunk = std::min<int64_t>(chunk, (g->slots + o.force_windows - 1) / o.force_windows);
    chunk = std::max<int64_t>(chunk, 1 << 16);
    const int64_t max_row = [&]() {
      int64_t m = 0;
      for (int64_t i = 0; i < n; ++i) m = std::max<int64_t>(m, g->h_ptr[i + 1] - g->h_ptr[i]);
      return m;
    }();
    chunk = std::max(chunk, max_row);
    uint32_t* stage = sc.alloc<uint32_t>(chunk);
    if (!stage) return GS_ENOMEM;
    for (int64_t h0 = 0; h0 < n;) {
      int64_t h1 = h0;
      while (h1 < n && g->h_ptr[h1 + 1] - g->h_ptr[h0] <= chunk) ++h1;
      const int64_t off = g->h_ptr[h0];
      const int64_t words = g->h_ptr[h1] - off;
      timer.start(s);
      { rows_fill<<<row_blocks, kCellThreads, cell_smem, s>>>(g->d_xyzp, G, ncell, start, cnt,
                                                             g->d_edges2, nb, g->d_deg, g->d_ptr,
                                                             stage, h0, h1, off, kCellCap); note_launch(); }
      timer.stop(s);
      { k_graph_stats<<<grid_blocks((h1 - h0) * 32, 256), 256, 0, s>>>(g->d_deg, g->d_ptr, stage, off, h0, h1,
                                                                     tot, tot + 1, (int*)(tot + 2)); note_launch(); }
      ce = cudaMemcpyAsync(g->h_adj + off, stage, sizeof(uint32_t) * words, cudaMemcpyDeviceToHost, s);
      if (ce != cudaSuccess) return cuda_status(ce);
      ce = cudaStreamSynchronize(s);  // the staging buffer is reused
      if (ce != cudaSuccess) return cuda_status(ce);
      h0 = h1;
    }
    std::vector<int32_t> hdeg(n);
    cudaMemcpy(hdeg.data(), g->d_deg, sizeof(int32_t) * n, cudaMemcpyDeviceToHost);
    // first id of the last x-slab (cells are x-major); open boxes: n
    g->wrap_start = n;
    if (box_u) {
      int32_t ws = 0;
      const int64_t c_last = (int64_t)(G.nc[0] - 1) * G.nc[1] * G.nc[2];
      cudaMemcpy(&ws, start + c_last, sizeof(int32_t), cudaMemcpyDeviceToHost);
      g->wrap_start = ws;
    }
    g->h_reach.resize(n);
    g->h_far.assign(n, 0);
    for (int64_t i = 0; i < n; ++i) {
      const uint32_t* r = g->h_adj + g->h_ptr[i];
      int d = hdeg[i];
      if (i < g->wrap_start) {  // split off the wrap-around neighbours
        int e = d;
        while (e > 0 && (int64_t)edge_id(r[e - 1]) >= g->wrap_start) --e;
        g->h_far[i] = (e < d) ? 1 : 0;
        d = e;
      }
      g->h_reach[i] = d ? (int32_t)edge_id(r[d - 1]) : (int32_t)i;
    }
    WindowPlan plan;
    st = plan_windows(*g, o, &plan, 0, n);
    if (st) return st;
    g->windows = (int)plan.h0.size();
  }
  unsigned long long ht[3];
  cudaMemcpyAsync(ht, tot, sizeof(ht), cudaMemcpyDeviceToHost, s);
  ce = cudaStreamSynchronize(s);
  if (ce != cudaSuccess) return cuda_status(ce);
  g->probe_words = (int64_t)ht[0];
  g->edges_total = (int64_t)ht[1];
  g->max_deg = (int)(ht[2] & 0xffffffffu);
  g->h_deg.resize(n);
  ce = cudaMemcpy(g->h_deg.data(), g->d_deg, sizeof(int32_t) * n, cudaMemcpyDeviceToHost);
  if (ce != cudaSuccess) return cuda_status(ce);
  timer.publish();
  return cuda_status(cudaGetLastError());
}

namespace {
// walk[i] summed: for each edge (i, j), the words of N+(j) with id <= the
// largest id of N+(i).
__global__ void k_walk_words(const int32_t* __restrict__ deg, const int64_t* __restrict__ ptr,
                             const uint32_t* __restrict__ adj, int64_t adj_off, int64_t split,
                             int64_t adj_off2, int64_t h0, int64_t h1,
                             unsigned long long* total) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  unsigned long long acc = 0;
  for (int64_t i = h0 + blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < h1;
       i += warps) {
    const int d = deg[i];
    if (d == 0) continue;
    const uint32_t* r = row_at(adj, ptr, i, adj_off, split, adj_off2);
    const uint32_t hub_hi = edge_id(r[d - 1]);
    for (int k = lane; k < d; k += 32) {
      const uint32_t j = edge_id(r[k]);
      const uint32_t* rj = row_at(adj, ptr, j, adj_off, split, adj_off2);
      int lo = 0, hi = deg[j];
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (edge_id(rj[mid]) <= hub_hi) lo = mid + 1;
        else hi = mid;
      }
      acc += (unsigned long long)lo;
    }
  }
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) atomicAdd(total, acc);
}
}  // namespace

namespace {
// Triangles (i < j < k) and the sum over them of |N+(k)|: one warp per hub,
// lanes over the words of each spoke row N+(j); a word k is a triangle when
// a binary search finds it in N+(i).
__global__ void k_tri_words(const int32_t* __restrict__ deg, const int64_t* __restrict__ ptr,
                            const uint32_t* __restrict__ adj, int64_t adj_off, int64_t split,
                            int64_t adj_off2, int64_t h0, int64_t h1, unsigned long long* tri,
                            unsigned long long* words) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  unsigned long long nt = 0, nw = 0;
  for (int64_t i = h0 + blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < h1;
       i += warps) {
    const int d = deg[i];
    if (d < 2) continue;
    const uint32_t* r = row_at(adj, ptr, i, adj_off, split, adj_off2);
    for (int s = 0; s + 1 < d; ++s) {
      const uint32_t j = edge_id(r[s]);
      const uint32_t* rj = row_at(adj, ptr, j, adj_off, split, adj_off2);
      const int dj = deg[j];
      for (int t = lane; t < dj; t += 32) {
        const uint32_t k = edge_id(rj[t]);
        int lo = s + 1, hi = d;  // k > j, so only the hub row after j
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (edge_id(r[mid]) < k) lo = mid + 1;
          else hi = mid;
        }
        if (lo < d && edge_id(r[lo]) == k) {
          nt += 1;
          nw += (unsigned long long)deg[k];
        }
      }
    }
  }
  for (int o = 16; o; o >>= 1) {
    nt += __shfl_xor_sync(0xffffffffu, nt, o);
    nw += __shfl_xor_sync(0xffffffffu, nw, o);
  }
  if (lane == 0) {
    atomicAdd(tri, nt);
    atomicAdd(words, nw);
  }
}
}  // namespace

int tri_words_device(const Graph& g, int64_t* tri, int64_t* words) {
  *tri = *words = 0;
  if (g.n == 0 || g.slots == 0) return GS_OK;
  Opts o;
  Scratch sc(o.stream);
  unsigned long long* tot = sc.alloc<unsigned long long>(2);
  if (!tot) return GS_ENOMEM;
  cudaMemsetAsync(tot, 0, 2 * sizeof(unsigned long long), o.stream);
  int st = for_each_window(g, o, sc, [&](const WinView& v) -> int {
    { k_tri_words<<<grid_blocks((v.h1 - v.h0) * 32, 256), 256, 0, o.stream>>>(
        g.d_deg, g.d_ptr, v.adj, v.off1, v.split, v.off2, v.h0, v.h1, tot, tot + 1); note_launch(); }
    return cuda_status(cudaGetLastError());
  });
  if (st) return st;
  unsigned long long h[2] = {0, 0};
  cudaMemcpyAsync(h, tot, sizeof(h), cudaMemcpyDeviceToHost, o.stream);
  cudaError_t e = cudaStreamSynchronize(o.stream);
  if (e != cudaSuccess) return cuda_status(e);
  *tri = (int64_t)h[0];
  *words = (int64_t)h[1];
  return GS_OK;
}

int walk_words_device(Graph* g) {
  if (g->n == 0 || g->slots == 0) {
    g->walk_words = 0;
    return GS_OK;
  }
  Opts o;
  Scratch sc(o.stream);
  unsigned long long* tot = sc.alloc<unsigned long long>(1);
  if (!tot) return GS_ENOMEM;
  cudaMemsetAsync(tot, 0, sizeof(unsigned long long), o.stream);
  int st = for_each_window(*g, o, sc, [&](const WinView& v) -> int {
    { k_walk_words<<<grid_blocks((v.h1 - v.h0) * 32, 256), 256, 0, o.stream>>>(
        g->d_deg, g->d_ptr, v.adj, v.off1, v.split, v.off2, v.h0, v.h1, tot); note_launch(); }
    return cuda_status(cudaGetLastError());
  });
  if (st) return st;
  unsigned long long h = 0;
  cudaMemcpyAsync(&h, tot, sizeof(h), cudaMemcpyDeviceToHost, o.stream);
  cudaError_t e = cudaStreamSynchronize(o.stream);
  if (e != cudaSuccess) return cuda_status(e);
  g->walk_words = (int64_t)h;
  return GS_OK;
}

void shard_range(const Graph& g, const Opts& o, int64_t* lo, int64_t* hi) {
  *lo = 0;
  *hi = g.n;
  if (o.shards <= 1 || g.n == 0) return;
  // boundaries at equal shares of the edge words (h_ptr is nondecreasing)
  const int64_t total = g.h_ptr[g.n];
  auto bound = [&](int k) -> int64_t {
    if (k <= 0) return 0;
    if (k >= o.shards) return g.n;
    const int64_t target = (int64_t)((__int128)total * k / o.shards);
    return std::lower_bound(g.h_ptr.begin(), g.h_ptr.begin() + g.n, target) - g.h_ptr.begin();
  };
  *lo = bound(o.shard);
  *hi = bound(o.shard + 1);
}

int plan_windows(const Graph& g, const Opts& o, WindowPlan* plan, int64_t lo, int64_t hi) {
  const std::vector<int64_t>& P = g.h_ptr;
  const int64_t n = g.n, ws = g.wrap_start;
  const int64_t far_words = P[n] - P[ws];
  // a query without its own budget / window count uses the graph's
  const uint64_t budget = o.budget ? o.budget : g.budget;
  const int force = o.force_windows > 0 ? o.force_windows : g.force_windows;
  const int64_t cap = budget ? (int64_t)(budget / (2 * sizeof(uint32_t))) : INT64_MAX;
  const int64_t target = force > 0 ? (P[hi] - P[lo] + force - 1) / force : INT64_MAX;
  // words a window [h0, h1) with near reach r and far flag f needs
  auto need = [&](int64_t h0, int64_t r, bool f) -> int64_t {
    if (f && r >= ws) return P[n] - P[h0];  // the two ranges touch: one range
    return (P[r] - P[h0]) + (f ? far_words : 0);
  };
  plan->h0.clear();
  plan->h1.clear();
  plan->r1.clear();
  plan->far.clear();
  plan->max_words = 0;
  int64_t h0 = lo;
  while (h0 < hi) {
    int64_t h1 = h0, reach = h0 + 1;
    bool far = false;
    while (h1 < hi) {
      const int64_t nr =
          std::max<int64_t>(std::max<int64_t>(reach, (int64_t)g.h_reach[h1] + 1), h1 + 1);
      const bool nf = far || g.h_far[h1];
      const int64_t own = P[h1 + 1] - P[h0];
      if (h1 > h0 && (own > target || need(h0, nr, nf) > cap)) break;
      reach = nr;
      far = nf;
      ++h1;
    }
    const int64_t words = need(h0, reach, far);
    if (words > cap) return GS_ENOMEM;  // one hub's rows exceed a window buffer
    if (far && reach >= ws) {
      reach = n;
      far = false;
    }
    plan->h0.push_back(h0);
    plan->h1.push_back(h1);
    plan->r1.push_back(reach);
    plan->far.push_back(far ? 1 : 0);
    plan->max_words = std::max(plan->max_words, words);
    h0 = h1;
  }
  return GS_OK;
}

}  // namespace gs
