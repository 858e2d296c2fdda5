// Configuration tooling on the binned counts: the Cayley-Menger
// realisability mask of the 4pCF orbits (Sec. 5.2) and exact fine-to-coarse
// rebinning of 3pCF and parity 4pCF results (Sec. 5.1).
//
// The mask evaluates 144 V^2 from the six squared edge lengths in 128-bit
// integers on doubled bin centres, so its sign is exact. Rebinning maps
// every fine configuration to its coarse one (or drops it), sorts the fine
// indices stably by target and then sums each target's fine entries in
// ascending fine order: integer channels are exact and the FP64 channels
// are reproducible from run to run.
#include <algorithm>

#include "gs_internal.cuh"

namespace gs {
namespace {

// 144 V^2 from squared edges in slot order (01, 02, 03, 12, 13, 23): with
// opposite pairs (01, 23), (02, 13), (03, 12) and the four faces
// (01, 02, 12), (01, 03, 13), (02, 03, 23), (12, 13, 23).
__device__ inline __int128 volume2_x144(const int64_t* p) {
  const __int128 a = p[0], b = p[1], c = p[2], f = p[3], e = p[4], d = p[5];
  return a * d * (b + c + e + f - a - d) + b * e * (a + c + d + f - b - e) +
         c * f * (a + b + d + e - c - f) - a * b * f - a * c * e - b * c * d - d * e * f;
}

__global__ void k_cm_mask(const uint8_t* __restrict__ reps, int64_t n_orbits,
                          const int64_t* __restrict__ c2, uint8_t* mask,
                          unsigned long long* kept) {
  unsigned local = 0;
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n_orbits;
       o += (int64_t)gridDim.x * blockDim.x) {
    int64_t p[6];
#pragma unroll
    for (int s = 0; s < 6; ++s) p[s] = c2[reps[6 * o + s]];
    const uint8_t m = volume2_x144(p) > 0 ? 1 : 0;
    mask[o] = m;
    local += m;
  }
  for (int off = 16; off; off >>= 1) local += __shfl_xor_sync(0xffffffffu, local, off);
  if ((threadIdx.x & 31) == 0 && local) atomicAdd(kept, (unsigned long long)local);
}

// Fine 3pCF configuration -> coarse index (or -1), one thread per sorted
// fine triple.
__global__ void k_rebin3_targets(int nbf, const int32_t* __restrict__ map, int nbc,
                                 int32_t* target, int8_t* sign) {
  const int64_t raw_n = (int64_t)nbf * nbf * nbf;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < raw_n;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(r / ((int64_t)nbf * nbf)), y = (int)((r / nbf) % nbf), z = (int)(r % nbf);
    if (!(x <= y && y <= z)) continue;
    const int f = conf3_rank(x, y, z, nbf);
    const int mx = map[x], my = map[y], mz = map[z];
    target[f] = (mx < 0 || my < 0 || mz < 0) ? -1 : conf3_rank(mx, my, mz, nbc);
    sign[f] = 1;
  }
}

// Fine 4pCF orbit -> coarse orbit (or -1) and the sign an odd count takes:
// the fine representative's bins go through the map in its own vertex
// labelling; the coarse table gives the orbit and whether the relabelling
// onto the coarse representative is odd. Coarse orbits that are not chiral
// take no odd part (sign 0).
__global__ void k_rebin4_targets(const uint8_t* __restrict__ reps_f, int64_t nf,
                                 const int32_t* __restrict__ map, const uint32_t* __restrict__ lut_c,
                                 int nbc, int32_t* target, int8_t* sign) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf;
       f += (int64_t)gridDim.x * blockDim.x) {
    int m[6];
    bool drop = false;
#pragma unroll
    for (int s = 0; s < 6; ++s) {
      m[s] = map[reps_f[6 * f + s]];
      drop |= m[s] < 0;
    }
    if (drop) {
      target[f] = -1;
      sign[f] = 0;
      continue;
    }
    // table digit order (b01, b02, b12, b03, b13, b23) from slot order
    const int64_t k = (((((int64_t)m[0] * nbc + m[1]) * nbc + m[3]) * nbc + m[2]) * nbc + m[4]) * nbc + m[5];
    const uint32_t ent = lut_c[k];
    target[f] = (int32_t)(ent & 0x3FFFFFFFu);
    sign[f] = (ent >> 31) ? (((ent >> 30) & 1u) ? -1 : 1) : 0;
  }
}

__global__ void k_target_counts(const int32_t* __restrict__ target, int64_t nf, int32_t* cnt) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf;
       f += (int64_t)gridDim.x * blockDim.x)
    if (target[f] >= 0) atomicAdd(cnt + target[f], 1);
}

// Stable placement of the fine indices by target: one warp walks the fine
// indices in order, 32 at a time; lanes with equal targets take consecutive
// slots in lane (= fine index) order.
__global__ void k_stable_fill(const int32_t* __restrict__ target, int64_t nf,
                              const int32_t* __restrict__ off, int32_t* cursor, int32_t* list) {
  const int lane = threadIdx.x;
  for (int64_t base = 0; base < nf; base += 32) {
    const int64_t f = base + lane;
    const int t = f < nf ? target[f] : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, t);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    if (t >= 0) {
      const int pos = off[t] + cursor[t] + rank;
      list[pos] = (int32_t)f;
    }
    __syncwarp();
    if (t >= 0 && rank == 0) cursor[t] += __popc(peers);
    __syncwarp();
  }
}

// Sum each coarse configuration's fine entries in ascending fine order.
__global__ void k_rebin_sum(const int32_t* __restrict__ off, const int32_t* __restrict__ list,
                            const int8_t* __restrict__ sign, int64_t nc,
                            const unsigned long long* __restrict__ e_in, const long long* __restrict__ o_in,
                            const double* __restrict__ we_in, const double* __restrict__ wo_in,
                            unsigned long long* e_out, long long* o_out, double* we_out,
                            double* wo_out) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc;
       c += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long e = 0;
    long long o = 0;
    double we = 0.0, wo = 0.0;
    for (int k = off[c]; k < off[c + 1]; ++k) {
      const int f = list[k];
      const int s = sign[f];
      if (e_in) e += e_in[f];
      if (we_in) we = __dadd_rn(we, we_in[f]);
      if (s != 0) {
        if (o_in) o += s * o_in[f];
        if (wo_in) wo = __dadd_rn(wo, s > 0 ? wo_in[f] : -wo_in[f]);
      }
    }
    if (e_out) e_out[c] = e;
    if (o_out) o_out[c] = o;
    if (we_out) we_out[c] = we;
    if (wo_out) wo_out[c] = wo;
  }
}

int grid_for(int64_t n, int threads) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t need = (n + threads - 1) / threads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)sms * 8));
}

int check_map(const int32_t* bin_map, int nbf, int nbc, std::vector<int32_t>* host) {
  host->assign(nbf, 0);
  cudaPointerAttributes at;
  const bool on_dev = cudaPointerGetAttributes(&at, bin_map) == cudaSuccess &&
                      (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
  cudaGetLastError();
  if (on_dev) {
    if (cudaMemcpy(host->data(), bin_map, sizeof(int32_t) * nbf, cudaMemcpyDeviceToHost) != cudaSuccess)
      return GS_ECUDA;
  } else {
    std::copy(bin_map, bin_map + nbf, host->begin());
  }
  for (int32_t v : *host)
    if (v < -1 || v >= nbc) return GS_EINVAL;
  return GS_OK;
}

struct RebinIo {
  const void* in[4];
  void* out[4];
  size_t in_elem[4];
};

// Shared tail of both rebinning calls: sort by target, sum, copy back.
int rebin_common(int64_t nf, int64_t nc, int32_t* d_target, int8_t* d_sign, const RebinIo& io,
                 const Opts& o, Scratch& sc) {
  cudaStream_t s = o.stream;
  int32_t* cnt = sc.alloc<int32_t>(nc + 1);
  int32_t* cursor = sc.alloc<int32_t>(nc);
  int32_t* list = sc.alloc<int32_t>(std::max<int64_t>(nf, 1));
  if (!cnt || !cursor || !list) return GS_ENOMEM;
  cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (nc + 1), s);
  cudaMemsetAsync(cursor, 0, sizeof(int32_t) * nc, s);
  { k_target_counts<<<grid_for(nf, 256), 256, 0, s>>>(d_target, nf, cnt); note_launch(); }
  int st = scan_exclusive_i32(cnt, cnt, nc + 1, nullptr, s, sc);
  if (st) return st;
  { k_stable_fill<<<1, 32, 0, s>>>(d_target, nf, cnt, cursor, list); note_launch(); }
  const void* din[4];
  void* dout[4];
  for (int k = 0; k < 4; ++k) {
    din[k] = io.in[k] ? to_device(sc, io.in[k], io.in_elem[k] * nf, s) : nullptr;
    if (io.in[k] && !din[k]) return GS_ENOMEM;
    dout[k] = !io.out[k] ? nullptr
                         : (is_device_ptr(io.out[k]) ? io.out[k] : sc.alloc_bytes(8 * (size_t)nc));
    if (io.out[k] && !dout[k]) return GS_ENOMEM;
  }
  { k_rebin_sum<<<grid_for(nc, 256), 256, 0, s>>>(
      cnt, list, d_sign, nc, static_cast<const unsigned long long*>(din[0]),
      static_cast<const long long*>(din[1]), static_cast<const double*>(din[2]),
      static_cast<const double*>(din[3]), static_cast<unsigned long long*>(dout[0]),
      static_cast<long long*>(dout[1]), static_cast<double*>(dout[2]), static_cast<double*>(dout[3])); note_launch(); }
  st = cuda_status(cudaGetLastError());
  for (int k = 0; k < 4 && !st; ++k)
    if (io.out[k] && dout[k] != io.out[k])
      st = cuda_status(cudaMemcpyAsync(io.out[k], dout[k], 8 * (size_t)nc, cudaMemcpyDeviceToHost, s));
  cudaError_t e = cudaStreamSynchronize(s);
  if (!st) st = cuda_status(e);
  return st;
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" {

int gs_config_mask_cm(int nb, const int64_t* edges_u, uint8_t* mask, int64_t* n_realisable,
                      const gs_options* options) {
  if (!edges_u || !mask || nb < 1) return GS_EINVAL;
  if (nb > kMaxBins4) return GS_ERANGE;
  if (edges_u[0] < 0) return GS_EINVAL;
  for (int b = 0; b < nb; ++b)
    if (edges_u[b + 1] <= edges_u[b]) return GS_EINVAL;
  if (edges_u[nb] > (int64_t(1) << 19)) return GS_ERANGE;
  const Opts o = read_opts(options);
  int st = GS_OK;
  const Conf4Tables* t = conf4_tables(nb, &st);
  if (!t) return st;
  const int64_t no = t->n_orbits;
  std::vector<int64_t> c2(nb);
  for (int b = 0; b < nb; ++b) {
    const int64_t twice_centre = edges_u[b] + edges_u[b + 1];
    c2[b] = twice_centre * twice_centre;
  }
  {
    Scratch sc(o.stream);
    const int64_t* dc2 = static_cast<const int64_t*>(to_device(sc, c2.data(), sizeof(int64_t) * nb, o.stream));
    unsigned long long* kept = sc.alloc<unsigned long long>(1);
    uint8_t* dm = is_device_ptr(mask) ? mask : sc.alloc<uint8_t>(no);
    if (!dc2 || !kept || !dm) return GS_ENOMEM;
    cudaMemsetAsync(kept, 0, sizeof(unsigned long long), o.stream);
    { k_cm_mask<<<grid_for(no, 256), 256, 0, o.stream>>>(t->d_reps, no, dc2, dm, kept); note_launch(); }
    st = cuda_status(cudaGetLastError());
    if (!st && dm != mask)
      st = cuda_status(cudaMemcpyAsync(mask, dm, no, cudaMemcpyDeviceToHost, o.stream));
    unsigned long long h = 0;
    if (!st) st = cuda_status(cudaMemcpyAsync(&h, kept, sizeof(h), cudaMemcpyDeviceToHost, o.stream));
    cudaError_t e = cudaStreamSynchronize(o.stream);
    if (!st) st = cuda_status(e);
    if (!st && n_realisable) *n_realisable = (int64_t)h;
  }
  return st;
}

int gs_rebin_3pcf(int nb_fine, int nb_coarse, const int32_t* bin_map, const uint64_t* counts,
                  const double* wsum, uint64_t* coarse_counts, double* coarse_wsum,
                  const gs_options* options) {
  if (!bin_map || nb_fine < 1 || nb_coarse < 1) return GS_EINVAL;
  if (nb_fine > kMaxBins || nb_coarse > kMaxBins) return GS_ERANGE;
  if ((counts == nullptr) != (coarse_counts == nullptr) || (wsum == nullptr) != (coarse_wsum == nullptr))
    return GS_EINVAL;
  std::vector<int32_t> hmap;
  int st = check_map(bin_map, nb_fine, nb_coarse, &hmap);
  if (st) return st;
  const Opts o = read_opts(options);
  const int64_t nf = num_conf3(nb_fine), nc = num_conf3(nb_coarse);
  Scratch sc(o.stream);
  const int32_t* dmap = static_cast<const int32_t*>(to_device(sc, hmap.data(), sizeof(int32_t) * nb_fine, o.stream));
  int32_t* target = sc.alloc<int32_t>(nf);
  int8_t* sign = sc.alloc<int8_t>(nf);
  if (!dmap || !target || !sign) return GS_ENOMEM;
  const int64_t raw = (int64_t)nb_fine * nb_fine * nb_fine;
  { k_rebin3_targets<<<grid_for(raw, 256), 256, 0, o.stream>>>(nb_fine, dmap, nb_coarse, target, sign); note_launch(); }
  RebinIo io = {{counts, nullptr, wsum, nullptr},
                {coarse_counts, nullptr, coarse_wsum, nullptr},
                {8, 8, 8, 8}};
  return rebin_common(nf, nc, target, sign, io, o, sc);
}

int gs_rebin_4pcf(int nb_fine, int nb_coarse, const int32_t* bin_map, const uint64_t* even,
                  const int64_t* odd, const double* weven, const double* wodd, uint64_t* c_even,
                  int64_t* c_odd, double* c_weven, double* c_wodd, const gs_options* options) {
  if (!bin_map || nb_fine < 1 || nb_coarse < 1) return GS_EINVAL;
  if (nb_fine > kMaxBins4 || nb_coarse > kMaxBins4) return GS_ERANGE;
  if ((even == nullptr) != (c_even == nullptr) || (odd == nullptr) != (c_odd == nullptr) ||
      (weven == nullptr) != (c_weven == nullptr) || (wodd == nullptr) != (c_wodd == nullptr))
    return GS_EINVAL;
  std::vector<int32_t> hmap;
  int st = check_map(bin_map, nb_fine, nb_coarse, &hmap);
  if (st) return st;
  const Opts o = read_opts(options);
  const Conf4Tables* tf = conf4_tables(nb_fine, &st);
  if (!tf) return st;
  const Conf4Tables* tc = conf4_tables(nb_coarse, &st);
  if (!tc) return st;
  const int64_t nf = tf->n_orbits, nc = tc->n_orbits;
  Scratch sc(o.stream);
  const int32_t* dmap = static_cast<const int32_t*>(to_device(sc, hmap.data(), sizeof(int32_t) * nb_fine, o.stream));
  int32_t* target = sc.alloc<int32_t>(nf);
  int8_t* sign = sc.alloc<int8_t>(nf);
  if (!dmap || !target || !sign) return GS_ENOMEM;
  { k_rebin4_targets<<<grid_for(nf, 256), 256, 0, o.stream>>>(tf->d_reps, nf, dmap, tc->d_lut, nb_coarse,
                                                              target, sign); note_launch(); }
  RebinIo io = {{even, odd, weven, wodd}, {c_even, c_odd, c_weven, c_wodd}, {8, 8, 8, 8}};
  return rebin_common(nf, nc, target, sign, io, o, sc);
}

}  // extern "C"
