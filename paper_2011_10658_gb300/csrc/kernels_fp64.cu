// FP64 SIMT kernels: grouped K-concatenated GEMM with optional row gathers,
// Lanczos vector reductions, per-sector Cholesky, tridiagonal eigensolver.
// GB300's FP64 rate is a small fraction of its tensor throughput, so these
// kernels are simple register-tiled DFMA loops; the mixed-precision path
// replaces the hot contraction with tensor-core kernels.
#include <cfloat>
#include <atomic>
#include <type_traits>
#include <cstdio>

#include "kernels.cuh"

namespace qed {

static std::atomic<long long> g_launches{0};
long long launch_count() { return g_launches.load(); }
void count_launches(int n) { g_launches += n; }

namespace {

constexpr int BK = 16;
constexpr int THREADS = 256;

// FP64 -> FP32 with round-to-nearest-even, done on the integer pipes from the
// IEEE-754 formats (sign, rebiased exponent, top 23 of the 52 fraction bits,
// rounding on the 29 dropped bits; a carry out of the fraction bumps the
// exponent, up to infinity).  Magnitudes below the FP32 normal range become
// signed zero, NaN stays NaN.  GB300 runs FP64 instructions, conversions
// included, at a small fraction of its FP32 rate, so the FP32 grouped GEMM
// converts its FP64 operands this way.
__device__ __forceinline__ float d2f_bits(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7ff);
  const unsigned long long frac = b & 0xFFFFFFFFFFFFFull;
  if (e == 0x7ff) return __uint_as_float(sign | 0x7f800000u | (frac ? 0x400000u : 0u));
  const int fe = e - 1023 + 127;
  if (fe <= 0) return __uint_as_float(sign);
  if (fe >= 255) return __uint_as_float(sign | 0x7f800000u);
  unsigned r = sign | ((unsigned)fe << 23) | (unsigned)(frac >> 29);
  const unsigned rem = (unsigned)(frac & 0x1FFFFFFFull);
  if (rem > 0x10000000u || (rem == 0x10000000u && (r & 1u))) r += 1u;
  return __uint_as_float(r);
}

// FP32 -> FP64, exact, on the integer pipes (FP32 subnormals become zero).
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  const int e = (int)((u >> 23) & 0xff);
  const unsigned long long frac = u & 0x7FFFFFu;
  if (e == 0) return __longlong_as_double((long long)sign);
  if (e == 0xff) return __longlong_as_double((long long)(sign | 0x7FF0000000000000ull | (frac << 29)));
  return __longlong_as_double((long long)(sign | ((unsigned long long)(e - 127 + 1023) << 52) | (frac << 29)));
}

// ---- float-float arithmetic: a value hi + lo held in two FP32 numbers
// (about 48 significant bits), with products and sums made error-free by
// FMA (Dekker's TwoProduct) and Knuth's TwoSum.  GB300 runs FP32 at many
// times its FP64 rate, so a float-float multiply-add (about a dozen FP32
// instructions) outruns one FP64 FMA while keeping FP64-level accuracy for
// these contractions.
struct ff {
  float hi, lo;
  __device__ __forceinline__ ff() {}
  __device__ __forceinline__ explicit ff(float h) : hi(h), lo(0.f) {}
  __device__ __forceinline__ ff(float h, float l) : hi(h), lo(l) {}
};

__device__ __forceinline__ ff ff_norm(float s, float e) {
  const float h = s + e;
  return ff(h, e - (h - s));
}

__device__ __forceinline__ ff operator*(ff a, ff b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return ff_norm(p, e);
}

__device__ __forceinline__ ff operator+(ff a, ff b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  const float err = (a.hi - (s - bb)) + (b.hi - bb) + a.lo + b.lo;
  return ff_norm(s, err);
}

__device__ __forceinline__ ff& operator*=(ff& a, ff b) { a = a * b; return a; }
__device__ __forceinline__ ff& operator+=(ff& a, ff b) { a = a + b; return a; }

// c + a b with the product's error and the sum's error kept in lo
__device__ __forceinline__ ff kc_fma(ff a, ff b, ff c) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const float s = c.hi + p;
  const float bb = s - c.hi;
  const float err = (c.hi - (s - bb)) + (p - bb);
  return ff(s, c.lo + e + err);
}

__device__ __forceinline__ double kc_fma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float kc_fma(float a, float b, float c) { return fmaf(a, b, c); }

// FP64 -> float-float on the integer pipes: hi = the double cut to 24
// significant bits, lo = the remaining 29 fraction bits (rounded to 24)
__device__ __forceinline__ ff d2ff(double d);

template <typename T>
__device__ __forceinline__ T to_t(double v);
template <>
__device__ __forceinline__ double to_t<double>(double v) { return v; }
template <>
__device__ __forceinline__ float to_t<float>(double v) { return d2f_bits(v); }

template <>
__device__ __forceinline__ ff to_t<ff>(double v) { return d2ff(v); }

__device__ __forceinline__ ff d2ff(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const float hi = d2f_bits(__longlong_as_double((long long)(b & ~((1ull << 29) - 1ull))));
  const int e = (int)((b >> 52) & 0x7ff);
  const unsigned low = (unsigned)(b & ((1ull << 29) - 1ull));
  float lo = 0.f;
  if (e != 0 && e != 0x7ff && low) {
    // low x 2^(e - 1075): convert the integer, then move its exponent
    const float f = (float)low;
    const int ex = (int)((__float_as_uint(f) >> 23) & 0xff) + (e - 1075);
    if (ex > 0) lo = __uint_as_float((__float_as_uint(f) & 0x807fffffu) | ((unsigned)ex << 23));
    if (b >> 63) lo = -lo;
  }
  return ff(hi, lo);
}

template <typename T>
__device__ __forceinline__ double to_d(T v);
template <>
__device__ __forceinline__ double to_d<double>(double v) { return v; }
template <>
__device__ __forceinline__ double to_d<float>(float v) { return f2d_bits(v); }
template <>
__device__ __forceinline__ double to_d<ff>(ff v) { return f2d_bits(v.hi) + f2d_bits(v.lo); }

// Row maps are sign-encoded: -1 = zero row, otherwise (row << 1) | negate.
// Arithmetic in T (FP64, or FP32 with the operands converted first).
template <typename T>
__device__ __forceinline__ T load_a(const KChunk& c, int m, int k) {
  long long row = m;
  T scale = T(1);
  if (c.amap) {
    int r = c.amap[m];
    if (r < 0) return T(0);
    row = r >> 1;
    if (r & 1) scale = T(-1);
  }
  if (c.aval) scale *= to_t<T>(c.aval[m]);
  return scale * to_t<T>(c.A[row * c.a_m + (long long)k * c.a_k]);
}

template <typename T>
__device__ __forceinline__ T load_b(const KChunk& c, int k, int n) {
  long long row = k;
  T scale = T(1);
  if (c.bmap) {
    int r = c.bmap[k];
    if (r < 0) return T(0);
    row = r >> 1;
    if (r & 1) scale = T(-1);
  }
  if (c.bval) scale *= to_t<T>(c.bval[k]);
  return scale * to_t<T>(c.B[row * c.b_k + (long long)n * c.b_n]);
}

// One CTA computes a BM x BN tile of one output (16 x 16 threads, each a
// BM/16 x BN/16 register tile) over its chunk range, K staged in slabs of 16.
template <typename T, int BM, int BN>
__global__ void __launch_bounds__(THREADS) kc_gemm_kernel(const KTile* __restrict__ tiles,
                                                           const KOutput* __restrict__ outs,
                                                           const KChunk* __restrict__ chunks,
                                                           double* __restrict__ scratch) {
  constexpr int TM = BM / 16, TN = BN / 16;
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const KTile tile = tiles[blockIdx.x];
  const KOutput out = outs[tile.out];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
  for (int ci = tile.chunk_begin; ci < tile.chunk_end; ++ci) {
    const KChunk c = chunks[ci];
    if (c.add) {
      // C[m,n] += alpha * A[m,n]
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          const int m = tile.m0 + ty * TM + i, n = tile.n0 + tx * TN + j;
          if (m < out.M && n < out.N) acc[i][j] += to_t<T>(c.alpha) * load_a<T>(c, m, n);
        }
      continue;
    }
    const T alpha = to_t<T>(c.alpha);
    for (int k0 = 0; k0 < c.K; k0 += BK) {
      for (int e = tid; e < BM * BK; e += THREADS) {
        const int mm = e / BK, kk = e % BK;
        const int m = tile.m0 + mm, k = k0 + kk;
        As[kk][mm] = (m < out.M && k < c.K) ? alpha * load_a<T>(c, m, k) : T(0);
      }
      for (int e = tid; e < BN * BK; e += THREADS) {
        const int kk = e / BN, nn = e % BN;
        const int n = tile.n0 + nn, k = k0 + kk;
        Bs[kk][nn] = (n < out.N && k < c.K) ? load_b<T>(c, k, n) : T(0);
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        T a[TM], bv[TN];
#pragma unroll
        for (int i = 0; i < TM; ++i) a[i] = As[kk][ty * TM + i];
#pragma unroll
        for (int j = 0; j < TN; ++j) bv[j] = Bs[kk][tx * TN + j];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] = kc_fma(a[i], bv[j], acc[i][j]);
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int m = tile.m0 + ty * TM + i, n = tile.n0 + tx * TN + j;
      if (m >= out.M || n >= out.N) continue;
      const double v = to_d<T>(acc[i][j]);
      if (tile.part >= 0) {
        scratch[out.part_off + (long long)tile.part * out.M * out.N + (long long)m * out.N + n] = v;
      } else {
        double* p = out.C + (long long)m * out.c_m + (long long)n * out.c_n;
        *p = out.accumulate ? (*p + v) : v;
      }
    }
}

__global__ void kc_reduce_kernel(const KOutput* __restrict__ outs, const int* __restrict__ red_list,
                                 const double* __restrict__ scratch) {
  const KOutput out = outs[red_list[blockIdx.y]];
  const long long mn = (long long)out.M * out.N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < mn; e += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int p = 0; p < out.n_parts; ++p) s += scratch[out.part_off + p * mn + e];
    int m = (int)(e / out.N), n = (int)(e % out.N);
    double* c = out.C + (long long)m * out.c_m + (long long)n * out.c_n;
    *c = out.accumulate ? (*c + s) : s;
  }
}

// ------------------------------------------------------------ reductions
constexpr int RED_THREADS = 256;
constexpr int RED_BLOCKS = 304;   // 2 x 152 SMs
constexpr int LZ_BLOCKS = 1216;   // 8 x 152 SMs: the fused Lanczos passes keep GB300's FP64 pipes busy
constexpr int kMaxLz = 129;       // basis vectors a fused pass handles

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[RED_THREADS / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x < 32) {
    r = threadIdx.x < RED_THREADS / 32 ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  }
  return r;   // valid in thread 0
}

__global__ void dot_partial_kernel(const double* __restrict__ x, const double* __restrict__ y, long long n,
                                   double* __restrict__ partial) {
  double v = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    v = fma(x[i], y[i], v);
  v = block_sum(v);
  if (threadIdx.x == 0) partial[blockIdx.x] = v;
}

// Gate of a conditional reorthogonalisation pass (Daniel-Gragg-Kaufman-Stewart):
// the pass runs only if ||w||^2 after the first pass fell below ratio times
// ||w||^2 before it.
__device__ __forceinline__ bool gated_off(const double* num, const double* den, double ratio) {
  return num && *num >= ratio * *den;
}

__global__ void finish_kernel(const double* __restrict__ partial, int count, int stride, double* __restrict__ out,
                              const double* gate_num = nullptr, const double* gate_den = nullptr, double ratio = 0.0) {
  if (gated_off(gate_num, gate_den, ratio)) return;
  // blockIdx.x selects which vector of partials (multidot)
  double v = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) v += partial[(long long)blockIdx.x * stride + i];
  v = block_sum(v);
  if (threadIdx.x == 0) out[blockIdx.x] = v;
}

__global__ void multidot_partial_kernel(const double* __restrict__ Q, long long ldq, int k,
                                        const double* __restrict__ w, long long n, double* __restrict__ partial,
                                        const double* gate_num, const double* gate_den, double ratio) {
  if (gated_off(gate_num, gate_den, ratio)) return;
  // blockIdx.y = column j
  const int j = blockIdx.y;
  const double* q = Q + (long long)j * ldq;
  double v = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    v = fma(q[i], w[i], v);
  v = block_sum(v);
  if (threadIdx.x == 0) partial[(long long)j * gridDim.x + blockIdx.x] = v;
}

__global__ void multiaxpy_kernel(const double* __restrict__ Q, long long ldq, int k, const double* __restrict__ c,
                                 double* __restrict__ w, long long n, const double* gate_num, const double* gate_den,
                                 double ratio) {
  if (gated_off(gate_num, gate_den, ratio)) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double v = w[i];
    for (int j = 0; j < k; ++j) v = fma(-c[j], Q[(long long)j * ldq + i], v);
    w[i] = v;
  }
}

__global__ void combine_kernel(const double* __restrict__ Q, long long ldq, int k, const double* __restrict__ c,
                               double* __restrict__ x, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int j = 0; j < k; ++j) v = fma(c[j], Q[(long long)j * ldq + i], v);
    x[i] = v;
  }
}

// ---- fused Lanczos reorthogonalisation (one pass per Gram-Schmidt step)
// Second classical Gram-Schmidt pass wanted (Daniel-Gragg-Kaufman-Stewart)?
// The norm left after the first pass (*mid) against half the norm of the
// three-term residual (c1[k] = w'.w').
__device__ __forceinline__ bool lz_second_pass(const double* c1, int k, const double* mid, double ratio) {
  return *mid < ratio * c1[k];
}

// With alpha != NULL (first pass): y <- w' = y - alpha v_a - beta v_b (the
// three-term recurrence; v_b optional), written back.  Then
// partial[col * gridDim.x + block] for col < k: V_col . w' over this block's
// rows; col = k: w' . w'.  Columns in groups of eight per sweep over the
// rows (each thread visits the same rows in every sweep, so it reads back
// its own w').  With c1 != NULL the kernel runs only when a second pass is
// wanted.
// FF: products and sums in float-float arithmetic on the FP32 pipes (FP64
// data; GB300's FP64 pipes would otherwise bound these passes).
template <bool FF>
__global__ void lz_dots_kernel(const double* __restrict__ V, long long ldq, int k, double* __restrict__ y,
                               long long n, double* __restrict__ partial, const double* alpha,
                               const double* __restrict__ va, const double* beta, const double* __restrict__ vb,
                               const double* c1, const double* mid, double ratio) {
  if (c1 && !lz_second_pass(c1, k, mid, ratio)) return;
  __shared__ double sh[8][RED_THREADS / 32];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const double a = alpha ? *alpha : 0.0;
  const double b = (alpha && vb) ? *beta : 0.0;
  using A = typename std::conditional<FF, ff, double>::type;
  for (int g0 = 0; g0 <= k; g0 += 8) {
    A acc[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) acc[t] = A(0.f);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
      double yi = y[i];
      if (alpha && g0 == 0) {
        yi = fma(-a, va[i], yi);
        if (vb) yi = fma(-b, vb[i], yi);
        y[i] = yi;
      }
      const A ya = to_t<A>(yi);
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int col = g0 + t;
        if (col < k) acc[t] = kc_fma(to_t<A>(V[(long long)col * ldq + i]), ya, acc[t]);
        else if (col == k) acc[t] = kc_fma(ya, ya, acc[t]);
      }
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      double v = to_d<A>(acc[t]);
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (l == 0) sh[t][w] = v;
    }
    __syncthreads();
    if (threadIdx.x < 8 && g0 + (int)threadIdx.x <= k) {
      double v = 0.0;
      for (int u = 0; u < RED_THREADS / 32; ++u) v += sh[threadIdx.x][u];
      partial[(long long)(g0 + threadIdx.x) * gridDim.x + blockIdx.x] = v;
    }
    __syncthreads();
  }
}

// out[col] = sum of partial[col * count ..] (col = blockIdx.x).  Same gate as
// lz_dots_kernel.
__global__ void lz_finish_kernel(const double* __restrict__ partial, int count, double* __restrict__ out,
                                 const double* c1, int k1, const double* mid, double ratio) {
  if (c1 && !lz_second_pass(c1, k1, mid, ratio)) return;
  double v = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) v += partial[(long long)blockIdx.x * count + i];
  v = block_sum(v);
  if (threadIdx.x == 0) out[blockIdx.x] = v;
}

// y -= sum_{col < k} c[col] V_col, and partial[block] = this block's part of
// |y|^2 afterwards.  Same gate as lz_dots_kernel.
template <bool FF>
__global__ void lz_axpy_norm_kernel(const double* __restrict__ V, long long ldq, int k, const double* __restrict__ c,
                                    double* __restrict__ y, long long n, double* __restrict__ partial,
                                    const double* c1, const double* mid, double ratio) {
  if (c1 && !lz_second_pass(c1, k, mid, ratio)) return;
  using A = typename std::conditional<FF, ff, double>::type;
  __shared__ A cs[kMaxLz];
  for (int j = threadIdx.x; j < k; j += blockDim.x) cs[j] = to_t<A>(-c[j]);
  __syncthreads();
  A acc = A(0.f);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    A v = to_t<A>(y[i]);
    for (int j = 0; j < k; ++j) v = kc_fma(cs[j], to_t<A>(V[(long long)j * ldq + i]), v);
    y[i] = to_d<A>(v);
    acc = kc_fma(v, v, acc);
  }
  const double r = block_sum(to_d<A>(acc));
  if (threadIdx.x == 0) partial[blockIdx.x] = r;
}

// v = y / sqrt(nrm2), beta = sqrt(nrm2), *nrm_out = nrm2, with nrm2 the norm
// after the second pass when it ran, else after the first.
__global__ void lz_normalize_kernel(const double* __restrict__ y, double* __restrict__ v, long long n,
                                    const double* c1, int k1, const double* mid, const double* nrm_second,
                                    double ratio, double* beta, double* nrm_out) {
  const double nrm2 = lz_second_pass(c1, k1, mid, ratio) ? *nrm_second : *mid;
  const double inv = 1.0 / sqrt(nrm2);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    v[i] = y[i] * inv;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *beta = sqrt(fmax(nrm2, 0.0));
    *nrm_out = nrm2;
  }
}

__global__ void sqrt_kernel(const double* in, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) out[0] = sqrt(fmax(in[0], 0.0));
}

__global__ void axpby_kernel(const double* __restrict__ x, double* __restrict__ y, long long n, const double* a_dev,
                             double a_const, double a_sign, const double* b_dev, double b_const) {
  const double a = a_sign * (a_dev ? *a_dev : a_const);
  const double b = b_dev ? *b_dev : b_const;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = fma(a, x[i], b * y[i]);
}

__global__ void scale_inv_sqrt_kernel(const double* __restrict__ x, double* __restrict__ y, long long n,
                                      const double* nrm2) {
  const double inv = 1.0 / sqrt(*nrm2);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = x[i] * inv;
}

__global__ void copy_kernel(const double* __restrict__ x, double* __restrict__ y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = x[i];
}

__global__ void add_scaled_kernel(const double* __restrict__ x, double* __restrict__ y, long long n, double a) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = fma(a, x[i], y[i]);
}

__global__ void zero_kernel(double* __restrict__ x, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] = 0.0;
}

// flag = 1 if some x[i] is NaN or infinite (exponent field all ones).
__global__ void check_finite_kernel(const double* __restrict__ x, long long n, int* flag) {
  bool bad = false;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    bad |= ((__double_as_longlong(x[i]) >> 52) & 0x7ff) == 0x7ff;
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicExch(flag, 1);
}

__global__ void to_float_kernel(const double* __restrict__ x, float* __restrict__ y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}

__global__ void to_double_kernel(const float* __restrict__ x, double* __restrict__ y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (double)x[i];
}

// SplitMix64 (Steele, Lea & Flood 2014), counter form: output i (1-based)
// is mix(seed + i * gamma); value 2 * (x >> 11) * 2^-53 - 1.
__global__ void fill_uniform_kernel(double* __restrict__ x, long long n, uint64_t seed, uint64_t start) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    uint64_t z = seed + (start + (uint64_t)i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    x[i] = 2.0 * (double)(z >> 11) * 0x1.0p-53 - 1.0;
  }
}

// Upper Cholesky G = R^T R in shared memory, then R^{-1} by back substitution.
// One CTA per matrix; n <= 256.
__global__ void cholesky_inv_kernel(double* G, double* Rinv, const long long* off, const int* nn, const int* ldd,
                                    int* status, double ill_cond) {
  extern __shared__ double sh[];
  const int idx = blockIdx.x;
  const int n = nn[idx], ld = ldd[idx];
  double* g = G + off[idx];
  double* ri = Rinv + off[idx];
  double* R = sh;                // n x n
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) R[e] = g[(e / n) * ld + (e % n)];
  __syncthreads();
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  // largest original diagonal = squared largest column norm of the factored matrix
  __shared__ double gmax;
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int j = 0; j < n; ++j) mx = fmax(mx, R[j * n + j]);
    gmax = mx;
  }
  __syncthreads();
  // right-looking: for column j, R[j][j] = sqrt(G[j][j]), R[j][i] = G[j][i]/R[j][j], trailing update
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      double d = R[j * n + j];
      if (!(d > 0.0)) { bad = 1; d = 1.0; }
      else if (d <= ill_cond * gmax) bad = bad ? bad : 2;
      R[j * n + j] = sqrt(d);
    }
    __syncthreads();
    const double rjj = R[j * n + j];
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) R[j * n + i] /= rjj;
    __syncthreads();
    for (int e = threadIdx.x; e < (n - j - 1) * (n - j - 1); e += blockDim.x) {
      int a = j + 1 + e / (n - j - 1), b = j + 1 + e % (n - j - 1);
      if (b >= a) R[a * n + b] -= R[j * n + a] * R[j * n + b];
    }
    __syncthreads();
  }
  // write R (upper) back to G, zero below
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    int a = e / n, b = e % n;
    g[a * ld + b] = b >= a ? R[e] : 0.0;
  }
  __syncthreads();
  // Rinv: solve R X = I column by column (thread per column)
  for (int col = threadIdx.x; col < n; col += blockDim.x) {
    for (int a = n - 1; a >= 0; --a) {
      double v = (a == col) ? 1.0 : 0.0;
      for (int b = a + 1; b <= col; ++b) v -= R[a * n + b] * ri[b * ld + col];
      ri[a * ld + col] = (a <= col) ? v / R[a * n + a] : 0.0;
    }
    for (int a = col + 1; a < n; ++a) ri[a * ld + col] = 0.0;
  }
  if (threadIdx.x == 0) status[idx] = bad;
}


// Classical Gram-Schmidt applied twice per column, one CTA per sector matrix
// (column-major m x n at X + xoff, Q written in place, R (n x n) at
// R + roff with leading dimension ldr).  A column whose remainder is at
// most dep_tol * (largest column norm) is dependent: R_jj = 0 and q_j is
// the first unit vector e_k (k increasing, never reused) whose remainder
// after two projections exceeds accept.
constexpr int QR_THREADS = 1024;

__device__ double cta_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    double r = l < (int)(blockDim.x / 32) ? red[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    if (l == 0) red[32] = r;
  }
  __syncthreads();
  return red[32];
}

// c[i] = <q_i, v> for i < j (warp per i), then v -= sum_i c[i] q_i.
__device__ void project_out(const double* X, long long m, int j, double* v, double* c, double* Rcol) {
  const int w = threadIdx.x / 32, l = threadIdx.x % 32, nw = blockDim.x / 32;
  for (int i = w; i < j; i += nw) {
    const double* q = X + (long long)i * m;
    double acc = 0.0;
    for (long long r = l; r < m; r += 32) acc = fma(q[r], v[r], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (l == 0) c[i] = acc;
  }
  __syncthreads();
  for (long long r = threadIdx.x; r < m; r += blockDim.x) {
    double a = v[r];
    for (int i = 0; i < j; ++i) a = fma(-c[i], X[(long long)i * m + r], a);
    v[r] = a;
  }
  if (Rcol)
    for (int i = threadIdx.x; i < j; i += blockDim.x) Rcol[i] += c[i];
  __syncthreads();
}

__global__ void __launch_bounds__(QR_THREADS) cgs2_qr_kernel(double* X, const long long* xoff, const int* rows,
                                                              const int* cols, double* R, const long long* roff,
                                                              int ldr, double dep_tol, double accept) {
  __shared__ double red[40];
  __shared__ double c[256];
  __shared__ double rcol[256];
  const int sidx = blockIdx.x;
  const long long m = rows[sidx];
  const int n = cols[sidx];
  double* x = X + xoff[sidx];
  double* Rs = R + roff[sidx];
  double scale = 0.0;
  for (int j = 0; j < n; ++j) {
    double acc = 0.0;
    for (long long r = threadIdx.x; r < m; r += blockDim.x) acc = fma(x[j * m + r], x[j * m + r], acc);
    scale = fmax(scale, sqrt(cta_sum(acc, red)));
  }
  long long next_k = 0;
  for (int j = 0; j < n; ++j) {
    double* v = x + (long long)j * m;
    for (int i = threadIdx.x; i < n; i += blockDim.x) rcol[i] = 0.0;
    __syncthreads();
    project_out(x, m, j, v, c, rcol);
    project_out(x, m, j, v, c, rcol);
    double acc = 0.0;
    for (long long r = threadIdx.x; r < m; r += blockDim.x) acc = fma(v[r], v[r], acc);
    const double nv = sqrt(cta_sum(acc, red));
    if (nv > dep_tol * scale) {
      const double inv = 1.0 / nv;
      for (long long r = threadIdx.x; r < m; r += blockDim.x) v[r] *= inv;
      if (threadIdx.x == 0) rcol[j] = nv;
    } else {
      if (threadIdx.x == 0) rcol[j] = 0.0;
      // completion by unit vectors
      for (; next_k < m; ++next_k) {
        for (long long r = threadIdx.x; r < m; r += blockDim.x) v[r] = (r == next_k) ? 1.0 : 0.0;
        __syncthreads();
        project_out(x, m, j, v, c, nullptr);
        project_out(x, m, j, v, c, nullptr);
        double a2 = 0.0;
        for (long long r = threadIdx.x; r < m; r += blockDim.x) a2 = fma(v[r], v[r], a2);
        const double nw = sqrt(cta_sum(a2, red));
        if (nw > accept) {
          const double inv = 1.0 / nw;
          for (long long r = threadIdx.x; r < m; r += blockDim.x) v[r] *= inv;
          ++next_k;
          break;
        }
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) Rs[(long long)i * ldr + j] = i <= j ? rcol[i] : 0.0;
    __syncthreads();
  }
}

// ------------------------------------------------------------ tridiagonal
// Lowest eigenpair of the k x k symmetric tridiagonal T (diagonal a, squared
// off-diagonal b2) of a Lanczos cycle.  The leading principal minors
// p_i(x) = det(T_i - x I) obey p_i = (a_i - x) p_{i-1} - b2_{i-1} p_{i-2};
// the number of sign changes along p_0 = 1, p_1, .., p_k is the number of
// eigenvalues below x (Sturm).  Every operation is a multiply-add, so a warp
// evaluates 32 counts at once; the state is rescaled by exact powers of two.
constexpr int TRI_MAX = 128;
constexpr int RESTART_MAX = 8;   // Ritz vectors kept by a thick restart

__device__ __forceinline__ int dexp(double v) { return (__double2hiint(v) >> 20) & 0x7ff; }

// exact rescaling of the recurrence state (p, pm[, d, dm]) by 2^-512 / 2^512
__device__ __forceinline__ void rescale2(double& p, double& pm) {
  const int e = dexp(p);
  if (e > 1023 + 512) {
    p *= 0x1p-512; pm *= 0x1p-512;
  } else if (e < 1023 - 512 && dexp(pm) < 1023 - 512) {
    p *= 0x1p+512; pm *= 0x1p+512;
  }
}

__device__ int sturm_minors(const double* a, const double* b2, int k, double x) {
  double pm = 1.0, p = a[0] - x;
  int neg = __double2hiint(p) < 0 && p != 0.0;
  int cnt = neg;
  for (int i = 1; i < k; ++i) {
    const double pn = fma(a[i] - x, p, -b2[i - 1] * pm);
    const int nn = __double2hiint(pn) < 0 && pn != 0.0;   // zero counts as positive
    cnt += nn ^ neg;
    neg = nn;
    pm = p;
    p = pn;
    rescale2(p, pm);
  }
  return cnt;
}

// -p_{k-1}(x) / p_k'(x): the squared last component of the unit eigenvector
// of an eigenvalue x (ratio of the minor below to the derivative).
__device__ double last_component_sq(const double* a, const double* b2, int k, double x) {
  if (k == 1) return 1.0;
  double pm = 1.0, p = a[0] - x, dm = 0.0, d = -1.0;
  for (int i = 1; i < k; ++i) {
    const double t = a[i] - x;
    const double pn = fma(t, p, -b2[i - 1] * pm);
    const double dn = fma(t, d, -fma(b2[i - 1], dm, p));
    pm = p; p = pn; dm = d; d = dn;
    const int e = dexp(p) > dexp(d) ? dexp(p) : dexp(d);
    if (e > 1023 + 512) {
      p *= 0x1p-512; pm *= 0x1p-512; d *= 0x1p-512; dm *= 0x1p-512;
    } else if (e < 1023 - 512 && dexp(pm) < 1023 - 512 && dexp(dm) < 1023 - 512) {
      p *= 0x1p+512; pm *= 0x1p+512; d *= 0x1p+512; dm *= 0x1p+512;
    }
  }
  const double r = d != 0.0 ? -pm / d : 1.0;
  return fmin(fmax(r, 0.0), 1.0);
}

// Eigenvector of T for the eigenvalue theta: inverse iteration with a shift
// just below theta, tridiagonal LU (Thomas), orthogonalised against the
// n_prev rows of prev (stride ld) (vectors of lower eigenvalues of a
// cluster).  x normalised, x[0] >= 0 when n_prev == 0.
__device__ void inverse_iteration(const double* a, const double* b, int k, double theta, double scale, int iters,
                                  double* x, const double* prev, int ld, int n_prev) {
  double cp[TRI_MAX], dp[TRI_MAX];
  const double shift = theta - 1e-13 * fmax(scale, 1e-300) - 1e-300;
  for (int i = 0; i < k; ++i) x[i] = n_prev == 0 ? 1.0 : 1.0 + 0.37 * (double)(i % (n_prev + 2));
  for (int it = 0; it < iters; ++it) {
    double denom = a[0] - shift;
    if (denom == 0.0) denom = 1e-300;
    cp[0] = (k > 1 ? b[0] : 0.0) / denom;
    dp[0] = x[0] / denom;
    for (int i = 1; i < k; ++i) {
      double m = (a[i] - shift) - b[i - 1] * cp[i - 1];
      if (m == 0.0) m = 1e-300;
      const double inv = 1.0 / m;
      cp[i] = (i < k - 1 ? b[i] : 0.0) * inv;
      dp[i] = (x[i] - b[i - 1] * dp[i - 1]) * inv;
    }
    x[k - 1] = dp[k - 1];
    for (int i = k - 2; i >= 0; --i) x[i] = dp[i] - cp[i] * x[i + 1];
    for (int pass = 0; pass < 2; ++pass)
      for (int q = 0; q < n_prev; ++q) {
        double h = 0.0;
        for (int i = 0; i < k; ++i) h += prev[q * ld + i] * x[i];
        for (int i = 0; i < k; ++i) x[i] -= h * prev[q * ld + i];
      }
    double nrm = 0.0;
    for (int i = 0; i < k; ++i) nrm += x[i] * x[i];
    const double inv = 1.0 / sqrt(nrm);
    for (int i = 0; i < k; ++i) x[i] *= inv;
  }
  if (n_prev == 0 && x[0] < 0.0)
    for (int i = 0; i < k; ++i) x[i] = -x[i];
}

// Warp-collective multisection for the eigenvalue of index idx (0 = lowest):
// on entry [lo, hi] holds it (count(lo) <= idx < count(hi)); each round the 32
// lanes count at 32 interior points and the bracket shrinks 33-fold, until it
// is a few ulps wide.  All lanes return the same bracket.
__device__ void multisect(const double* a, const double* b2, int k, int idx, double& lo, double& hi) {
  const int lane = threadIdx.x & 31;
  for (int round = 0; round < 64; ++round) {
    const double w = hi - lo;
    if (w <= 4.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) + 1e-300) break;
    const double x = lo + w * ((double)(lane + 1) * (1.0 / 33.0));
    const unsigned above = __ballot_sync(0xffffffffu, sturm_minors(a, b2, k, x) > idx);
    double nlo, nhi;
    if (above == 0u) {
      nlo = __shfl_sync(0xffffffffu, x, 31);
      nhi = hi;
    } else {
      const int f = __ffs(above) - 1;
      nhi = __shfl_sync(0xffffffffu, x, f);
      const double xl = __shfl_sync(0xffffffffu, x, f > 0 ? f - 1 : 0);
      nlo = f > 0 ? xl : lo;
    }
    if (!(nhi - nlo < w)) break;   // no progress left at this precision
    lo = nlo;
    hi = nhi;
  }
}

// Warp-collective: stage (a, b, b2) of the tridiagonal in shared memory and
// return its Gershgorin bracket (widened) and scale.
__device__ void stage_tridiag(const double* alpha, const double* beta, int k, double* a, double* b, double* b2,
                              double& lo, double& hi, double& scale) {
  const int lane = threadIdx.x & 31;
  for (int i = lane; i < k; i += 32) {
    a[i] = alpha[i];
    const double bi = i < k - 1 ? beta[i] : 0.0;
    b[i] = bi;
    b2[i] = bi * bi;
  }
  __syncwarp();
  lo = 1e300;
  hi = -1e300;
  for (int i = lane; i < k; i += 32) {
    const double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + fabs(b[i]);
    lo = fmin(lo, a[i] - r);
    hi = fmax(hi, a[i] + r);
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  const double span = hi - lo;
  scale = fmax(fabs(lo), fabs(hi));
  lo -= 1e-12 * span + 1e-300;
  hi += 1e-12 * span + 1e-300;
}

// One warp.  out[0] = theta (lowest eigenvalue), out[1] = |beta[k-1]| |s_k|
// (the Ritz residual estimate).  With want_vec the eigenvector goes to s and
// out[0] is its Rayleigh quotient; the vector is also formed when s_k is
// too small for the minor ratio to resolve.
__global__ void __launch_bounds__(32) tridiag_lowest_kernel(const double* __restrict__ alpha,
                                                            const double* __restrict__ beta, int k, double* out,
                                                            double* s, int want_vec) {
  __shared__ double a[TRI_MAX], b[TRI_MAX], b2[TRI_MAX];
  double lo, hi, scale;
  stage_tridiag(alpha, beta, k, a, b, b2, lo, hi, scale);
  multisect(a, b2, k, 0, lo, hi);
  if (threadIdx.x != 0) return;
  const double theta = 0.5 * (lo + hi);
  double sk = sqrt(last_component_sq(a, b2, k, theta));
  double th = theta;
  if (want_vec || sk < 1e-4) {
    double x[TRI_MAX];
    inverse_iteration(a, b, k, theta, scale, want_vec ? 3 : 2, x, nullptr, 0, 0);
    sk = fabs(x[k - 1]);
    if (want_vec) {
      double rq = 0.0;
      for (int i = 0; i < k; ++i) {
        double v = a[i] * x[i];
        if (i > 0) v += b[i - 1] * x[i - 1];
        if (i < k - 1) v += b[i] * x[i + 1];
        rq += x[i] * v;
      }
      th = rq;
      for (int i = 0; i < k; ++i) s[i] = x[i];
    }
  }
  out[0] = th;
  out[1] = fabs(beta[k - 1]) * sk;
}

// Thick restart of a Lanczos cycle (Wu and Simon's thick-restart Lanczos).
// From the k x k tridiagonal T (alpha, beta; beta[k-1] couples the residual
// vector r) keep the m lowest Ritz pairs (theta_i, s_i).  Their couplings to
// r are c_i = beta[k-1] s_i[k-1].  A Lanczos process on diag(theta) started
// from c / |c| gives an orthogonal U (m x p) and a p x p tridiagonal; in
// reversed order the kept vectors Z = V S U form a tridiagonal block whose
// last vector alone couples to r with |c|, so the next cycle continues the
// ordinary three-term recurrence from r at position p.  Writes C = S U
// reversed (k x p, row-major: C[r * p + i]), alpha[0..p), beta[0..p) (beta[p-1]
// = |c|) and *p_out.  One warp; serial parts in lane 0.
__global__ void __launch_bounds__(32) lanczos_restart_kernel(double* alpha, double* beta, int k, int m, double* C,
                                                             int* p_out) {
  __shared__ double a[TRI_MAX], b[TRI_MAX], b2[TRI_MAX];
  __shared__ double S[RESTART_MAX][TRI_MAX];
  __shared__ double th[RESTART_MAX];
  double glo, ghi, scale;
  stage_tridiag(alpha, beta, k, a, b, b2, glo, ghi, scale);
  if (m > k) m = k;
  for (int i = 0; i < m; ++i) {
    double lo = glo, hi = ghi;
    multisect(a, b2, k, i, lo, hi);
    if (threadIdx.x == 0) th[i] = 0.5 * (lo + hi);
  }
  __syncwarp();
  if (threadIdx.x != 0) return;
  const double bk = beta[k - 1];
  double c[RESTART_MAX];
  for (int i = 0; i < m; ++i) {
    inverse_iteration(a, b, k, th[i], scale, 3, S[i], &S[0][0], TRI_MAX, i);
    c[i] = bk * S[i][k - 1];
  }
  // Lanczos on diag(theta) from c / |c| with full reorthogonalisation
  double cn = 0.0;
  for (int i = 0; i < m; ++i) cn += c[i] * c[i];
  cn = sqrt(cn);
  double U[RESTART_MAX][RESTART_MAX];
  double la[RESTART_MAX], lb[RESTART_MAX];
  int p = 0;
  if (cn > 0.0) {
    for (int i = 0; i < m; ++i) U[0][i] = c[i] / cn;
    p = 1;
    for (int j = 0; j < m; ++j) {
      double w[RESTART_MAX];
      for (int i = 0; i < m; ++i) w[i] = th[i] * U[j][i];
      double aj = 0.0;
      for (int i = 0; i < m; ++i) aj += U[j][i] * w[i];
      la[j] = aj;
      for (int pass = 0; pass < 2; ++pass)
        for (int q = 0; q <= j; ++q) {
          double h = 0.0;
          for (int i = 0; i < m; ++i) h += U[q][i] * w[i];
          for (int i = 0; i < m; ++i) w[i] -= h * U[q][i];
        }
      double bj = 0.0;
      for (int i = 0; i < m; ++i) bj += w[i] * w[i];
      bj = sqrt(bj);
      if (j + 1 >= m || bj <= 1e-13 * fmax(scale, 1e-300)) break;
      lb[j] = bj;
      for (int i = 0; i < m; ++i) U[j + 1][i] = w[i] / bj;
      p = j + 2;
    }
  }
  if (p == 0) {   // r decoupled: keep the lowest Ritz vector alone
    p = 1;
    for (int i = 0; i < m; ++i) U[0][i] = i == 0 ? 1.0 : 0.0;
    la[0] = th[0];
  }
  // C[:, i] = S^T U[p-1-i] (reversed), new tridiagonal reversed
  for (int r = 0; r < k; ++r)
    for (int i = 0; i < p; ++i) {
      double v = 0.0;
      for (int q = 0; q < m; ++q) v += S[q][r] * U[p - 1 - i][q];
      C[r * p + i] = v;
    }
  for (int i = 0; i < p; ++i) alpha[i] = la[p - 1 - i];
  for (int i = 0; i + 1 < p; ++i) beta[i] = lb[p - 2 - i];
  beta[p - 1] = cn;
  *p_out = p;
}

// Z[:, i] = sum_r V[:, r] C[r * p + i] for i < p (p <= RESTART_MAX).
__global__ void rotate_basis_kernel(const double* __restrict__ V, long long ld, int k, const double* __restrict__ C,
                                    int p, double* __restrict__ Z, long long n) {
  __shared__ double cs[TRI_MAX * RESTART_MAX];
  for (int e = threadIdx.x; e < k * p; e += blockDim.x) cs[e] = C[e];
  __syncthreads();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double acc[RESTART_MAX];
#pragma unroll
    for (int q = 0; q < RESTART_MAX; ++q) acc[q] = 0.0;
    for (int r = 0; r < k; ++r) {
      const double v = V[(long long)r * ld + i];
#pragma unroll
      for (int q = 0; q < RESTART_MAX; ++q)
        if (q < p) acc[q] = fma(cs[r * p + q], v, acc[q]);
    }
#pragma unroll
    for (int q = 0; q < RESTART_MAX; ++q)
      if (q < p) Z[(long long)q * ld + i] = acc[q];
  }
}

int grid_for(long long n) {
  long long g = (n + 255) / 256;
  if (g > 152 * 8) g = 152 * 8;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

void launch_kc_gemm(const KTile* tiles, int n_tiles, const KOutput* outs, const KChunk* chunks, double* scratch,
                    cudaStream_t s, int fp32, int shape) {
  if (n_tiles <= 0) return;
#define QED_KC(T, BM, BN) kc_gemm_kernel<T, BM, BN><<<n_tiles, THREADS, 0, s>>>(tiles, outs, chunks, scratch)
#define QED_KC_ALL(T)                       \
  switch (shape) {                          \
    case KS_16: QED_KC(T, 16, 16); break;   \
    case KS_64: QED_KC(T, 64, 64); break;   \
    case KS_16x64: QED_KC(T, 16, 64); break; \
    case KS_64x16: QED_KC(T, 64, 16); break; \
    default: QED_KC(T, 32, 32); break;      \
  }
  if (fp32 == 1) {
    QED_KC_ALL(float)
  } else if (fp32 == 2) {
    QED_KC_ALL(ff)
  } else {
    QED_KC_ALL(double)
  }
#undef QED_KC_ALL
#undef QED_KC
  count_launches(1);
}

void launch_kc_reduce(const KOutput* outs, int n_outs, const int* red_list, int n_red, double* scratch,
                      cudaStream_t s) {
  if (n_red <= 0) return;
  dim3 grid(8, n_red);
  kc_reduce_kernel<<<grid, 256, 0, s>>>(outs, red_list, scratch);
  count_launches(1);
}

void launch_dot(const double* x, const double* y, long long n, double* partial, double* out, cudaStream_t s) {
  dot_partial_kernel<<<RED_BLOCKS, RED_THREADS, 0, s>>>(x, y, n, partial);
  count_launches(1);
  finish_kernel<<<1, RED_THREADS, 0, s>>>(partial, RED_BLOCKS, RED_BLOCKS, out);
  count_launches(1);
}

void launch_multidot(const double* Q, long long ldq, int k, const double* w, long long n, double* partial,
                     double* out, cudaStream_t s, const double* gate_num, const double* gate_den, double ratio) {
  if (k <= 0) return;
  dim3 grid(RED_BLOCKS, k);
  multidot_partial_kernel<<<grid, RED_THREADS, 0, s>>>(Q, ldq, k, w, n, partial, gate_num, gate_den, ratio);
  count_launches(1);
  finish_kernel<<<k, RED_THREADS, 0, s>>>(partial, RED_BLOCKS, RED_BLOCKS, out, gate_num, gate_den, ratio);
  count_launches(1);
}

void launch_multiaxpy(const double* Q, long long ldq, int k, const double* c, double* w, long long n,
                      cudaStream_t s, const double* gate_num, const double* gate_den, double ratio) {
  if (k <= 0) return;
  multiaxpy_kernel<<<grid_for(n), 256, 0, s>>>(Q, ldq, k, c, w, n, gate_num, gate_den, ratio);
  count_launches(1);
}

void launch_combine(const double* Q, long long ldq, int k, const double* c, double* x, long long n,
                    cudaStream_t s) {
  combine_kernel<<<grid_for(n), 256, 0, s>>>(Q, ldq, k, c, x, n);
  count_launches(1);
}

void launch_lz_reorth(const double* V, long long ldq, int k, double* y, long long n, double* partial, double* c1,
                      double* c2, double* mid, double* nrm_second, double ratio, double* alpha_j,
                      const double* beta_prev, double* beta_j, double* nrm_out, double* v_next, cudaStream_t s,
                      int ff_arith) {
  if (k < 1 || k >= kMaxLz) return;
  auto dots = ff_arith ? lz_dots_kernel<true> : lz_dots_kernel<false>;
  auto axpy = ff_arith ? lz_axpy_norm_kernel<true> : lz_axpy_norm_kernel<false>;
  const double* vj = V + (long long)(k - 1) * ldq;
  const double* vp = k >= 2 ? V + (long long)(k - 2) * ldq : nullptr;
  // alpha_j = v_j . y
  dot_partial_kernel<<<RED_BLOCKS, RED_THREADS, 0, s>>>(vj, y, n, partial);
  finish_kernel<<<1, RED_THREADS, 0, s>>>(partial, RED_BLOCKS, RED_BLOCKS, alpha_j);
  // first pass on w' = y - alpha_j v_j - beta_{j-1} v_{j-1}: c1 = V^T w',
  // c1[k] = w'.w'; y -= V c1; mid = |y|^2
  dots<<<LZ_BLOCKS, RED_THREADS, 0, s>>>(V, ldq, k, y, n, partial, alpha_j, vj, beta_prev, vp, nullptr,
                                                    nullptr, 0.0);
  lz_finish_kernel<<<k + 1, RED_THREADS, 0, s>>>(partial, LZ_BLOCKS, c1, nullptr, 0, nullptr, 0.0);
  axpy<<<LZ_BLOCKS, RED_THREADS, 0, s>>>(V, ldq, k, c1, y, n, partial, nullptr, nullptr, 0.0);
  lz_finish_kernel<<<1, RED_THREADS, 0, s>>>(partial, LZ_BLOCKS, mid, nullptr, 0, nullptr, 0.0);
  // second pass where the first removed more than the ratio allows
  dots<<<LZ_BLOCKS, RED_THREADS, 0, s>>>(V, ldq, k, y, n, partial, nullptr, nullptr, nullptr, nullptr, c1,
                                                    mid, ratio);
  lz_finish_kernel<<<k, RED_THREADS, 0, s>>>(partial, LZ_BLOCKS, c2, c1, k, mid, ratio);
  axpy<<<LZ_BLOCKS, RED_THREADS, 0, s>>>(V, ldq, k, c2, y, n, partial, c1, mid, ratio);
  lz_finish_kernel<<<1, RED_THREADS, 0, s>>>(partial, LZ_BLOCKS, nrm_second, c1, k, mid, ratio);
  lz_normalize_kernel<<<grid_for(n), 256, 0, s>>>(y, v_next, n, c1, k, mid, nrm_second, ratio, beta_j, nrm_out);
  count_launches(11);
}

void launch_sqrt(const double* in, double* out, cudaStream_t s) {
  sqrt_kernel<<<1, 32, 0, s>>>(in, out);
  count_launches(1);
}

void launch_axpby(const double* x, double* y, long long n, const double* a_dev, double a_const, double a_sign,
                  const double* b_dev, double b_const, cudaStream_t s) {
  axpby_kernel<<<grid_for(n), 256, 0, s>>>(x, y, n, a_dev, a_const, a_sign, b_dev, b_const);
  count_launches(1);
}

void launch_scale_inv_sqrt(const double* x, double* y, long long n, const double* nrm2, cudaStream_t s) {
  scale_inv_sqrt_kernel<<<grid_for(n), 256, 0, s>>>(x, y, n, nrm2);
  count_launches(1);
}

void launch_copy(const double* x, double* y, long long n, cudaStream_t s) {
  copy_kernel<<<grid_for(n), 256, 0, s>>>(x, y, n);
  count_launches(1);
}

void launch_fill_uniform(double* x, long long n, uint64_t seed, uint64_t start, cudaStream_t s) {
  if (n <= 0) return;
  fill_uniform_kernel<<<grid_for(n), 256, 0, s>>>(x, n, seed, start);
  count_launches(1);
}

void launch_add_scaled(const double* x, double* y, long long n, double a, cudaStream_t s) {
  add_scaled_kernel<<<grid_for(n), 256, 0, s>>>(x, y, n, a);
  count_launches(1);
}

void launch_zero(double* x, long long n, cudaStream_t s) {
  if (n <= 0) return;
  zero_kernel<<<grid_for(n), 256, 0, s>>>(x, n);
  count_launches(1);
}

void launch_check_finite(const double* x, long long n, int* flag, cudaStream_t s) {
  if (n <= 0) return;
  check_finite_kernel<<<grid_for(n), 256, 0, s>>>(x, n, flag);
  count_launches(1);
}

void launch_to_float(const double* x, float* y, long long n, cudaStream_t s) {
  to_float_kernel<<<grid_for(n), 256, 0, s>>>(x, y, n);
  count_launches(1);
}

void launch_to_double(const float* x, double* y, long long n, cudaStream_t s) {
  to_double_kernel<<<grid_for(n), 256, 0, s>>>(x, y, n);
  count_launches(1);
}

void launch_cholesky_inv(double* G, double* Rinv, const long long* off, const int* n, const int* ld, int count,
                         int max_n, double ill_cond, int* status, cudaStream_t s) {
  if (count <= 0) return;
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(cholesky_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 160 * 8);
    configured = true;
  }
  cholesky_inv_kernel<<<count, 256, (size_t)max_n * max_n * sizeof(double), s>>>(G, Rinv, off, n, ld, status,
                                                                                  ill_cond);
  count_launches(1);
}

void launch_cgs2_qr(double* X, const long long* xoff, const int* rows, const int* cols, int count, double* R,
                    const long long* roff, int ldr, double dep_tol, double accept, cudaStream_t s) {
  if (count <= 0) return;
  cgs2_qr_kernel<<<count, QR_THREADS, 0, s>>>(X, xoff, rows, cols, R, roff, ldr, dep_tol, accept);
  count_launches(1);
}

void launch_lanczos_restart(double* alpha, double* beta, int k, int m, double* C, int* p_out, cudaStream_t st) {
  if (k <= 0 || k > TRI_MAX || m < 1 || m > RESTART_MAX) return;
  lanczos_restart_kernel<<<1, 32, 0, st>>>(alpha, beta, k, m, C, p_out);
  count_launches(1);
}

void launch_rotate_basis(const double* V, long long ld, int k, const double* C, int p, double* Z, long long n,
                         cudaStream_t st) {
  if (k <= 0 || k > TRI_MAX || p < 1 || p > RESTART_MAX) return;
  rotate_basis_kernel<<<grid_for(n), 256, 0, st>>>(V, ld, k, C, p, Z, n);
  count_launches(1);
}

void launch_tridiag_lowest(const double* alpha, const double* beta, int k, double* out, double* s, int want_vec,
                           cudaStream_t st) {
  if (k <= 0 || k > TRI_MAX) return;
  tridiag_lowest_kernel<<<1, 32, 0, st>>>(alpha, beta, k, out, s, want_vec);
  count_launches(1);
}

}  // namespace qed
