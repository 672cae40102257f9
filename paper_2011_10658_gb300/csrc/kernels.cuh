// Device kernels of the TTN hot path (declarations shared by the engine).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace qed {

// Number of kernels launched by this library since load (all streams).
long long launch_count();
void count_launches(int n);

// One contribution A(MxK) * B(KxN) to an output.  Element addressing:
//   A[m,k] = sA * aval[m] * A[row*a_m + k*a_k],  amap[m] = (row << 1) | negate, -1 = zero row
//   B[k,n] = sB * bval[k] * B[row*b_k + n*b_n],  bmap[k] likewise (maps and vals optional)
// With add != 0 there is no B:  C[m,n] += alpha * A[m,n] (A[m,n] addressed as A[m,k=n]).
struct KChunk {
  const double* A;
  long long a_m, a_k;
  const int* amap;
  const double* aval;
  const double* B;
  long long b_k, b_n;
  const int* bmap;
  const double* bval;
  int K;
  int add;
  double alpha;
};

// An output C (MxN, C[m,n] at C + m*c_m + n*c_n) = sum of its chunks
// (accumulate != 0: C += sum).
struct KOutput {
  double* C;
  long long c_m, c_n;
  int M, N;
  int chunk_begin, chunk_end;
  int accumulate;
  int n_parts;        // > 1: split over chunk ranges, partial sums in scratch
  long long part_off; // scratch offset (doubles) of this output's partials
};

// One CTA's work: a BM x BN tile of an output over a chunk range.
struct KTile {
  int out;
  int m0, n0;
  int chunk_begin, chunk_end;
  int part;           // partial slot (-1: write C directly)
};

constexpr int KT_BM = 32;   // tile of the default shape
constexpr int KT_BN = 32;
// Tile shapes of the grouped GEMM (rows x columns of the output tile):
// 16x16, 32x32, 64x64, and the flat 16x64 / 64x16 for outputs with few rows
// (leg operators applied to a node tensor) or few columns.
enum KcShape { KS_16 = 0, KS_32 = 1, KS_64 = 2, KS_16x64 = 3, KS_64x16 = 4, KS_COUNT = 5 };
inline int kc_shape_m(int shape) {
  static const int m[KS_COUNT] = {16, 32, 64, 16, 64};
  return m[shape];
}
inline int kc_shape_n(int shape) {
  static const int n[KS_COUNT] = {16, 32, 64, 64, 16};
  return n[shape];
}

// fp32 = 1: same contraction with FP32 multiply-accumulate (operands
// rounded to FP32 on load, results stored as FP64); fp32 = 2: float-float
// arithmetic on the FP32 pipes (operands split into two FP32 numbers, about
// 48 significant bits; FP64-level accuracy).  shape: the tile shape the
// tiles were cut with.
void launch_kc_gemm(const KTile* tiles, int n_tiles, const KOutput* outs, const KChunk* chunks,
                    double* scratch, cudaStream_t s, int fp32 = 0, int shape = KS_32);
void launch_kc_reduce(const KOutput* outs, int n_outs, const int* red_list, int n_red, double* scratch,
                      cudaStream_t s);

// ---- vector kernels (FP64) ----
// partial sums per block then a single-block finish: deterministic.
void launch_dot(const double* x, const double* y, long long n, double* partial, double* out, cudaStream_t s);
// out[j] = <Q_j, w> for j < k (Q columns of length n, stride ldq).
// Optional gate (device scalars): the call does nothing when
// *gate_num >= ratio * *gate_den (a skipped reorthogonalisation pass).
void launch_multidot(const double* Q, long long ldq, int k, const double* w, long long n, double* partial,
                     double* out, cudaStream_t s, const double* gate_num = nullptr, const double* gate_den = nullptr,
                     double ratio = 0.0);
// w -= sum_j Q_j c[j]  (same optional gate)
void launch_multiaxpy(const double* Q, long long ldq, int k, const double* c, double* w, long long n,
                      cudaStream_t s, const double* gate_num = nullptr, const double* gate_den = nullptr,
                      double ratio = 0.0);
// x = sum_j c[j] Q_j
void launch_combine(const double* Q, long long ldq, int k, const double* c, double* x, long long n, cudaStream_t s);
// One Lanczos step after y = H v_{k-1} (V holds v_0 .. v_{k-1}, columns of
// stride ldq): alpha_j = v_j . y, the three-term residual
// w' = y - alpha_j v_j - beta_{j-1} v_{j-1} (beta_prev, unused for k = 1),
// classical Gram-Schmidt of w' against all k vectors (c1 = V^T w', w'.w' in
// c1[k]), a second pass into c2 when the Daniel-Gragg-Kaufman-Stewart test
// asks for it (decided on the device), then beta_j = |w|, *nrm_out = |w|^2
// and v_next = w / |w|.  Eleven launches; partial holds 1216 x (k + 1)
// doubles; c1 k + 1 and c2 k doubles; k <= 128.  ff_arith != 0: the dots and
// updates in float-float arithmetic on the FP32 pipes (about 2^-44 relative
// rounding per operation; the data stay FP64).
void launch_lz_reorth(const double* V, long long ldq, int k, double* y, long long n, double* partial, double* c1,
                      double* c2, double* mid, double* nrm_second, double ratio, double* alpha_j,
                      const double* beta_prev, double* beta_j, double* nrm_out, double* v_next, cudaStream_t s,
                      int ff_arith = 0);
// out[0] = sqrt(max(in[0], 0))
void launch_sqrt(const double* in, double* out, cudaStream_t s);
// y = a*x + b*y with a, b read from device scalars (nullable -> constants)
void launch_axpby(const double* x, double* y, long long n, const double* a_dev, double a_const, double a_sign,
                  const double* b_dev, double b_const, cudaStream_t s);
// y = x / sqrt(*nrm2) ; returns nothing
void launch_scale_inv_sqrt(const double* x, double* y, long long n, const double* nrm2, cudaStream_t s);
void launch_copy(const double* x, double* y, long long n, cudaStream_t s);
void launch_fill_uniform(double* x, long long n, uint64_t seed, uint64_t start, cudaStream_t s);
void launch_add_scaled(const double* x, double* y, long long n, double a, cudaStream_t s);
void launch_zero(double* x, long long n, cudaStream_t s);
void launch_to_float(const double* x, float* y, long long n, cudaStream_t s);
// *flag = 1 if any of x[0..n) is NaN or infinite (flag untouched otherwise).
void launch_check_finite(const double* x, long long n, int* flag, cudaStream_t s);
void launch_to_double(const float* x, double* y, long long n, cudaStream_t s);

// ---- small dense linear algebra (one CTA per matrix) ----
// For each matrix i: G_i (n_i x n_i at G + off_i, leading dim ld_i): in-place
// upper Cholesky R (G = R^T R) and then Rinv = R^{-1} (written to Rinv + off_i).
// status[i] = 0 ok, 1 non-positive pivot.
// status[i] = 2 when a pivot R_jj^2 <= ill_cond * max_j G_jj (ill-conditioned).
// max_n: largest n over the batch (<= 160).
void launch_cholesky_inv(double* G, double* Rinv, const long long* off, const int* n, const int* ld, int count,
                         int max_n, double ill_cond, int* status, cudaStream_t s);
// Gram-Schmidt QR (two passes per column) with deterministic completion of
// dependent columns; one CTA per column-major sector matrix (n <= 256).
void launch_cgs2_qr(double* X, const long long* xoff, const int* rows, const int* cols, int count, double* R,
                    const long long* roff, int ldr, double dep_tol, double accept, cudaStream_t s);

// Lowest eigenvalue of the symmetric tridiagonal (alpha[0..k), beta[0..k-1))
// (1 <= k <= 128).  out[0] = theta, out[1] = |beta[k-1] * s_k| (Ritz residual
// estimate; beta[k-1] is the trailing coupling).  With want_vec, s[0..k) gets
// the unit eigenvector (s[0] >= 0) and out[0] its Rayleigh quotient.
void launch_tridiag_lowest(const double* alpha, const double* beta, int k, double* out, double* svec, int want_vec,
                           cudaStream_t s);
// Thick restart (keep the m <= 8 lowest Ritz pairs of the k x k tridiagonal,
// k <= 128): writes the k x p combination C (row-major), the new leading
// p x p tridiagonal into alpha/beta with beta[p-1] the coupling to the
// residual vector, and p (1 <= p <= m) to *p_out.
void launch_lanczos_restart(double* alpha, double* beta, int k, int m, double* C, int* p_out, cudaStream_t s);
// Z[:, i] = sum_r V[:, r] C[r * p + i], i < p <= 8 (columns of length n, stride ld).
void launch_rotate_basis(const double* V, long long ld, int k, const double* C, int p, double* Z, long long n,
                         cudaStream_t s);

}  // namespace qed

namespace qed {

// ---- mixed-precision bottom-node H_eff (tcgen05) ----
// One output c-sector of y (rows x n, FP64, row-major with ld = n) is the
// sum of GEMM chunks  sign(r) * X[map(r), :] . W^T  accumulated in TMEM
// (A rows gathered into shared memory, B = W, both K-major) and of add terms
// alpha * sign(r) * val(r) * X32[map(r), :n] applied in FP32 in the epilogue.
struct TcChunk {
  const void* X;      // staging source sector matrix (BF16 or FP32), row stride xstride
  const int* map;     // sign-encoded row map (nullable: identity)
  const void* W;      // npad x kpad K-major B operand (alpha folded in)
  int kpad;           // K of the staged rows, multiple of 16 (split: [hi | lo], 2 x part)
  int xstride;        // elements per staged source row
};
struct TcAdd {
  const float* X32;   // FP32 staging source sector matrix, row stride ld
  const int* map;     // nullable: identity
  const double* val;  // nullable
  double alpha;
  int ld;
};
struct TcOutput {
  double* y;
  int rows, n, npad;
  int chunk_begin, chunk_end;
  int add_begin, add_end;
};
struct TcTile {
  int out;
  int row0;
};
// One conversion job: dst (rows x kpad, zero padded) <- scale * src (rows x cols, ld_src), FP64 source.
struct ConvJob {
  const double* src;
  long long ld_src;   // row stride of the source
  long long cs_src;   // column stride of the source
  void* dst;          // BF16 or FP32
  float* dst32;       // optional second FP32 copy (same padded layout)
  int rows, cols, kpad;
  double scale;
};

// elem: 2 = BF16 operands (kind::f16), 4 = TF32 operands (kind::tf32).
// split (TF32 only): A rows staged as [x_hi | x_lo] and B rows as [W_hi |
// W_lo]; three sub-products x_hi W_hi + x_hi W_lo + x_lo W_hi whose sum
// carries about 21 bits (x_lo W_lo dropped).
// err: device flag set to 1 if a wait timed out (results then invalid).
// polls: bound of each mbarrier wait in polls (< 0: the default, 2^22).
int launch_tc_heff(int elem, int split, const TcTile* tiles, int n_tiles, const TcOutput* outs,
                   const TcChunk* chunks, const TcAdd* adds, int max_kpad, int max_npad, int* err, cudaStream_t s,
                   long long polls = -1);
// ---- grouped leg contractions on the tensor cores (tcgen05) ----
// One contribution D[r, j] += alpha * sum_{k < K} A(r, k) B(j, k):
//   A(r, k) = A[(r / R2) * s1 + (r % R2) * s2 + k * sk]  (float if a_f32, else double)
//   B(j, k) = B[j * bj + k * bk]                          (double)
struct TgChunk {
  const void* A;
  long long s1, s2, sk;
  const double* B;
  long long bj, bk;
  int R2;
  int K;
  int a_f32;
  float alpha;
};
// An output: D[r, j] (r < rows, j < N) at C[(r / R2) * t1 + (r % R2) * t2 + j * cj],
// float if c_f32 (else double), written or added (accumulate); chunks of its
// tiles are summed in one accumulator; n_parts > 1: tiles write FP32 partial
// sums (rows x N each, at scratch + part_off) that the reduction adds up.
struct TgOut {
  void* C;
  long long t1, t2, cj;
  int R2;
  int rows, N, npad;
  int c_f32;
  int accumulate;
  int n_parts;
  long long part_off;
};
// One CTA: rows row0 .. row0 + 127 of output `out` over chunks [chunk_begin,
// chunk_end); part >= 0 writes partial slot `part`.
struct TgTile {
  int out;
  int row0;
  int chunk_begin, chunk_end;
  int part;
};
// Shared memory of one launch (two stages of A and B tiles).
int tg_stage_bytes(int elem, int split, int max_npad, int* a_bytes, int* b_bytes);
// elem 4: TF32 operands (split: three products of hi / lo parts), 2: BF16.
// red_list: outputs with n_parts > 1 (reduced after the GEMM).  err: device
// flag set if a wait timed out; polls < 0: default bound.
int launch_tg_gemm(int elem, int split, const TgTile* tiles, int n_tiles, const TgOut* outs, const TgChunk* chunks,
                   int max_npad, float* scratch, const int* red_list, int n_red, int* err, cudaStream_t s,
                   long long polls = -1);

// ---- FP64-accurate contractions on the BF16 tensor cores (digit planes) ----
constexpr int kOzDigits = 5;   // balanced base-256 digits per FP64 entry (about 2^-39 of the max)
// planes (16 bytes per entry, 8 BF16 planes of which kOzDigits are used)
// <- x[0..n), relative to 2^E >= max |x| (max |x| written to *amax).
void launch_oz_slice(const double* x, long long n, double* amax, void* planes, cudaStream_t s);
// Job: for one term and output sector, rows (c < cols) of the source sector
// matrix (at a_off, row stride a_ld, in planes) selected by map (sign-encoded
// source row per output row; NULL = identity).  Its FP64 partial blocks
// [part][c][c'] start at part_off.
struct OzJob {
  const int* map;
  long long a_off;
  long long part_off;
  int a_ld;
  int cols;
};
// CTA: jobs [job_begin, job_end) stacked in slots of `slot` MMA rows, against
// output sector rows [r0, r1) (at b_off, row stride b_ld, n columns c'),
// writing partial slot `part` of each job.
struct OzTile {
  long long b_off;
  int b_ld, n;
  int r0, r1;
  int job_begin, job_end;
  int slot;
  int part;
};
// One operator block O[c', c] (ld) += sum over its entries of alpha * the
// sum of that job's partial blocks.
struct OzSum {
  long long off;          // job's part_off
  long long part_stride;  // cols * n
  int n_parts;
  double alpha;
};
struct OzOut {
  double* O;
  int ld;
  int rows, cols;         // c' (output sector) x c (source sector)
  int sum_begin, sum_end;
};
// npad: MMA width (32 or 64, >= every tile's n).  err: set if a wait timed out.
int launch_oz_gram(const OzTile* tiles, int n_tiles, const OzJob* jobs, const void* planes, int npad, double* partial,
                   const OzOut* outs, int n_outs, const OzSum* sums, int* err, cudaStream_t s, long long polls = -1);

// mode 0: plain (BF16 or FP32 by elem); mode 1: split x rows [hi | lo] of
// width 2 kpad; mode 2: split W rows [hi | lo] of width 2 kpad.  hi is
// the value with its 13 low mantissa bits cleared (what the TF32 units read).
void launch_convert(int elem, int mode, const ConvJob* jobs, int n_jobs, long long max_elems, cudaStream_t s);

}  // namespace qed
