// Exact weighted sums for weights of wide dynamic range.
//
// The counting kernels sum products of fixed-point weights W (w = W 2^-S)
// exactly when |W| < 2^30. Weights whose magnitudes span more binades give
// larger W; for those every W is split exactly as W = A + 2^27 B with
// 0 <= A < 2^27 and |B| < 2^27 (|W| < 2^54). For an N-point statistic the
// wanted sum over tuples of prod_v W_v is the value at t = 2^27 of the
// polynomial P(t) = sum over tuples of prod_v (A_v + t B_v), of degree N.
// The kernels evaluate P exactly at N + 1 small points t (0, 1, -1, 2, -2),
// where |A + t B| < 2^29 keeps them on their exact path; its integer
// coefficients follow by exact interpolation and P(2^27) is assembled and
// rounded once to the nearest double. The coefficients come from an
// exactly solvable Vandermonde system:
//   degree 3 (t = 0, 1, -1, 2): c0 = P(0); with S(t) = P(t) - c0,
//     c2 = (S(1) + S(-1)) / 2, D = (S(1) - S(-1)) / 2 = c1 + c3,
//     E = (S(2) - 4 c2) / 2 = c1 + 4 c3, c3 = (E - D) / 3, c1 = D - c3;
//   degree 4 (t = 0, +-1, +-2): e1 = (P(1) + P(-1)) / 2 - c0 = c2 + c4,
//     o1 = (P(1) - P(-1)) / 2 = c1 + c3, e2 = (P(2) + P(-2)) / 2 - c0 =
//     4 c2 + 16 c4, o2 = (P(2) - P(-2)) / 2 = 2 c1 + 8 c3,
//     c4 = (e2 - 4 e1) / 12, c2 = e1 - c4, c3 = (o2 - 2 o1) / 6, c1 = o1 - c3.
// Every division is exact because the coefficients are integers.
#include <algorithm>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kSplitBits = 27;

__global__ void k_split_eval(const int64_t* __restrict__ W, int64_t n, int t, int64_t* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t w = W[i];
    const int64_t b = w >> kSplitBits;          // floor division
    const int64_t a = w - b * (int64_t(1) << kSplitBits);  // 0 <= a < 2^27
    out[i] = a + (int64_t)t * b;
  }
}

// Signed 320-bit integers, five 64-bit limbs, least significant first.
struct I320 {
  unsigned long long w[5];
};

__device__ inline I320 from192(const unsigned long long* p) {
  const unsigned long long ext = ((long long)p[2] < 0) ? ~0ull : 0ull;
  return I320{{p[0], p[1], p[2], ext, ext}};
}

__device__ inline I320 add(const I320& a, const I320& b) {
  I320 r;
  unsigned long long carry = 0;
  for (int k = 0; k < 5; ++k) {
    const unsigned long long s = a.w[k] + b.w[k];
    const unsigned long long c1 = s < a.w[k];
    r.w[k] = s + carry;
    carry = c1 | (r.w[k] < s);
  }
  return r;
}

__device__ inline I320 neg(const I320& a) {
  I320 r;
  unsigned long long carry = 1;
  for (int k = 0; k < 5; ++k) {
    r.w[k] = ~a.w[k] + carry;
    carry = (carry && r.w[k] == 0) ? 1ull : 0ull;
  }
  return r;
}

__device__ inline I320 sub(const I320& a, const I320& b) { return add(a, neg(b)); }

__device__ inline bool is_neg(const I320& a) { return (long long)a.w[4] < 0; }

// a * 2^s for 0 <= s < 64 (no overflow for the values met here)
__device__ inline I320 shl(const I320& a, int s) {
  if (s == 0) return a;
  I320 r;
  for (int k = 4; k >= 0; --k)
    r.w[k] = (a.w[k] << s) | (k ? a.w[k - 1] >> (64 - s) : 0ull);
  return r;
}

// a / d for a small d that divides a exactly (long division of the
// magnitude in 32-bit digits, so each step fits 64-bit arithmetic)
__device__ inline I320 div_exact(const I320& a, unsigned d) {
  const bool n = is_neg(a);
  const I320 m = n ? neg(a) : a;
  I320 q;
  unsigned long long rem = 0;
  for (int k = 4; k >= 0; --k) {
    const unsigned long long hi = (rem << 32) | (m.w[k] >> 32);
    const unsigned long long qh = hi / d;
    rem = hi % d;
    const unsigned long long lo = (rem << 32) | (m.w[k] & 0xFFFFFFFFull);
    const unsigned long long ql = lo / d;
    rem = lo % d;
    q.w[k] = (qh << 32) | ql;
  }
  return n ? neg(q) : q;
}

// value * 2^-scale to the nearest double, ties to even: the magnitude is
// rounded to odd at 64 significant bits, then converted by the hardware's
// round-to-nearest (two spare bits make the double rounding innocuous).
__device__ inline double to_double(const I320& a, int scale) {
  const bool n = is_neg(a);
  const I320 m = n ? neg(a) : a;
  int top = -1;
  for (int k = 4; k >= 0; --k)
    if (m.w[k]) {
      top = k;
      break;
    }
  if (top < 0) return 0.0;
  const int z = __clzll((long long)m.w[top]);
  unsigned long long win, lost = 0;
  int below;
  if (top == 0) {
    win = m.w[0];
    below = 0;
  } else {
    win = z ? (m.w[top] << z) | (m.w[top - 1] >> (64 - z)) : m.w[top];
    lost = z ? (m.w[top - 1] << z) : m.w[top - 1];
    for (int k = top - 2; k >= 0; --k) lost |= m.w[k];
    below = 64 * top - z;
  }
  win |= lost ? 1ull : 0ull;
  const double v = scalbn(__ull2double_rn(win), below - scale);
  return n ? -v : v;
}

// P: (degree + 1) blocks of n 192-bit sums, evaluated at 0, 1, -1, 2[, -2].
__global__ void k_combine(const unsigned long long* __restrict__ P, int64_t n, int degree,
                          int scale, double* out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const I320 p0 = from192(P + 3 * k);
    const I320 p1 = from192(P + 3 * (n + k));
    const I320 pm1 = from192(P + 3 * (2 * n + k));
    const I320 p2 = from192(P + 3 * (3 * n + k));
    I320 c[5];
    c[0] = p0;
    if (degree == 3) {
      const I320 s1 = sub(p1, p0), sm = sub(pm1, p0), s2 = sub(p2, p0);
      c[2] = div_exact(add(s1, sm), 2);
      const I320 D = div_exact(sub(s1, sm), 2);
      const I320 E = div_exact(sub(s2, shl(c[2], 2)), 2);
      c[3] = div_exact(sub(E, D), 3);
      c[1] = sub(D, c[3]);
      c[4] = I320{{0, 0, 0, 0, 0}};
    } else {
      const I320 pm2 = from192(P + 3 * (4 * n + k));
      const I320 e1 = sub(div_exact(add(p1, pm1), 2), p0);
      const I320 o1 = div_exact(sub(p1, pm1), 2);
      const I320 e2 = sub(div_exact(add(p2, pm2), 2), p0);
      const I320 o2 = div_exact(sub(p2, pm2), 2);
      c[4] = div_exact(sub(e2, shl(e1, 2)), 12);
      c[2] = sub(e1, c[4]);
      c[3] = div_exact(sub(o2, shl(o1, 1)), 6);
      c[1] = sub(o1, c[3]);
    }
    // P(2^27) by Horner: ((c4 2^27 + c3) 2^27 + c2) 2^27 + ...
    I320 v = c[degree];
    for (int m = degree - 1; m >= 0; --m) v = add(shl(v, kSplitBits), c[m]);
    out[k] = to_double(v, scale);
  }
}

const int kEvalPoints[5] = {0, 1, -1, 2, -2};

}  // namespace

int split_weights_device(const FixedW& fw, int64_t n, int t, int64_t* d_out, cudaStream_t s) {
  if (n > 0) {
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
    k_split_eval<<<blocks, 256, 0, s>>>(fw.d_W, n, t, d_out);
    note_launch();
  }
  return cuda_status(cudaGetLastError());
}

int combine_wide_device(const unsigned long long* d_P, int64_t n, int degree, int scale,
                        double* d_out, cudaStream_t s) {
  if (n > 0) {
    const int blocks = (int)std::min<int64_t>((n + 127) / 128, 1024);
    k_combine<<<blocks, 128, 0, s>>>(d_P, n, degree, scale, d_out);
    note_launch();
  }
  return cuda_status(cudaGetLastError());
}

int wide_eval_point(int k) { return kEvalPoints[k]; }

}  // namespace gs
