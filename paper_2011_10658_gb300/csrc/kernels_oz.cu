// FP64-accurate contractions on the BF16 tensor cores (Ozaki-type splitting).
//
// GB300 runs FP64 arithmetic at about 1 TFLOP/s, so the renormalized-operator
// updates at the bottom of the tree (Methods, "Tensor Networks": the
// operators of every term crossing the bond above a node, contracted with
// the node tensor T and its conjugate) are formed here on the BF16 tensor
// cores instead, at FP64-level accuracy:
//
//  * digit planes: every entry x of an FP64 array is written, relative to a
//    power of two 2^E >= max |x| of the array, as the integer
//    F = round(x 2^(W - E)), W = 8 S - 2, and F is split into S balanced
//    base-256 digits d_p in [-128, 127] (most significant first, which is
//    then at most 64 in magnitude); plane p
//    holds d_p 2^(E - W + 8 (S - 1 - p)) as a BF16 number (exact: a digit has
//    at most 8 significant bits).  The planes are stored interleaved, eight
//    BF16 values (16 bytes) per entry, S of them used.
//  * products: A B = sum_{p, q} A_p B_q; the pairs with p + q <= S - 1 are
//    kept (the rest lie below 2^-(8 S - 2) of |A| |B|).  All products of one
//    level l = p + q share one unit, and with |d| <= 128 a level's partial sum
//    over 128 K values and at most S pairs stays below 2^24 units, so the
//    tensor cores' FP32 accumulation is exact within such a slab.  Each level
//    has its own TMEM accumulator; after every slab the levels are added into
//    per-thread float-float (hi, lo) sums (Knuth's TwoSum), and the result is
//    written in FP64.
//
// oz_gram_kernel computes, for jobs j = (term, output sector), the blocks
//     D_j[c, c'] = sum_{r in K range} s_j(r) T_ic[src_j(r), c] T_oc[r, c'],
// i.e. one output sector's block of T^T (A (x) B) T for a term whose site
// operators A (x) B are a signed row selection (src_j, s_j) of the node
// tensor.  MMA rows are (job, c) pairs (up to four jobs of 32 columns per
// CTA), MMA columns c', K the rows r of the output sector, split into
// ranges over CTAs whose FP64 partial blocks are added afterwards by
// oz_reduce_kernel in a fixed order.  Both operands are staged transposed
// through registers: lane c of a warp reads entry (row, c) of eight rows
// (16 bytes each, all planes) and writes, per plane, the eight values as one
// 16-byte K chunk of row c.
#include <cuda_bf16.h>

#include <algorithm>

#include "kernels.cuh"

namespace qed {

namespace {

constexpr int OZ_THREADS = 128;
constexpr int OZ_KB = 32;                        // K rows per stage
constexpr int OZ_SLAB = 4;                       // stages per exact accumulation slab (128 K)
constexpr long long kOzWaitPolls = 1LL << 22;

__device__ __forceinline__ uint32_t oz_smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t oz_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

__device__ __forceinline__ uint32_t oz_core_off(int r, int q, int kchunks) {
  return (uint32_t)(((r >> 3) * kchunks + q) * 128 + (r & 7) * 16);
}

__device__ __forceinline__ bool oz_wait(uint32_t addr, uint32_t parity, long long polls) {
  for (long long it = 0; it < polls; ++it) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
    __nanosleep(32);
  }
  return false;
}

// Exponent E with max |x| < 2^E from the FP64 bits of max |x| (E = 0 for 0).
__device__ __forceinline__ int oz_scale_exp(double amax) {
  const long long b = __double_as_longlong(amax);
  const int e = (int)((b >> 52) & 0x7ff);
  return e == 0 ? 0 : e - 1022;   // amax < 2^(e - 1022)
}

// S balanced base-256 digits of x relative to 2^E, as BF16 plane values.
template <int S>
__device__ __forceinline__ uint4 oz_digits(double x, int E) {
  constexpr int W = 8 * S - 2;
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((bits >> 52) & 0x7ff);
  long long F = 0;
  if (e != 0 && e != 0x7ff) {
    const unsigned long long m = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    // x = m 2^(e - 1075); F = x 2^(W - E) = m 2^(e - 1075 + W - E)
    const int sh = 1075 - e - W + E;   // right shift (>= 1 when |x| < 2^E)
    unsigned long long f = 0;
    if (sh >= 64) f = 0;
    else if (sh >= 1) f = (m + (1ull << (sh - 1))) >> sh;
    else f = m << (-sh > 10 ? 10 : -sh);   // |x| >= 2^E: out of contract, clamped
    F = (bits >> 63) ? -(long long)f : (long long)f;
  }
  uint16_t h[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
  for (int p = S - 1; p >= 0; --p) {
    const int d = (int)(signed char)(F & 0xff);   // balanced digit in [-128, 127]
    F = (F - d) >> 8;
    // d 2^(E - W + 8 (S - 1 - p)) as BF16 (exact; zero stays zero)
    const int k = E - W + 8 * (S - 1 - p);
    float v = (float)d;
    if (d != 0) {
      // scale by 2^k in the exponent field; below the normal range -> 0
      const int ex = (int)((__float_as_uint(v) >> 23) & 0xff) + k;
      v = ex > 0 ? __uint_as_float(__float_as_uint(v) + ((unsigned)k << 23)) : 0.f;
    }
    const __nv_bfloat16 bv = __float2bfloat16_rz(v);
    h[p] = *(const uint16_t*)&bv;
  }
  uint4 out;
  out.x = (uint32_t)h[0] | ((uint32_t)h[1] << 16);
  out.y = (uint32_t)h[2] | ((uint32_t)h[3] << 16);
  out.z = (uint32_t)h[4] | ((uint32_t)h[5] << 16);
  out.w = (uint32_t)h[6] | ((uint32_t)h[7] << 16);
  return out;
}

template <int S>
__global__ void oz_slice_kernel(const double* __restrict__ x, long long n, const double* __restrict__ amax,
                                uint4* __restrict__ out) {
  const int E = oz_scale_exp(*amax);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = oz_digits<S>(x[i], E);
}

__global__ void oz_amax_kernel(const double* __restrict__ x, long long n, double* __restrict__ out) {
  __shared__ double sh[8];
  double v = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    // |x| on the integer pipes; max of non-negative doubles = max of their bits
    const long long b = __double_as_longlong(x[i]) & 0x7FFFFFFFFFFFFFFFll;
    v = __longlong_as_double(max(__double_as_longlong(v), b));
  }
  for (int o = 16; o > 0; o >>= 1)
    v = __longlong_as_double(max(__double_as_longlong(v), __double_as_longlong(__shfl_xor_sync(0xffffffffu, v, o))));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long m = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = max(m, __double_as_longlong(sh[w]));
    atomicMax((unsigned long long*)out, (unsigned long long)m);
  }
}

// plane p (0..7) of an interleaved entry
__device__ __forceinline__ uint32_t oz_plane(const uint4& v, int p) {
  const uint32_t w = p < 2 ? v.x : (p < 4 ? v.y : (p < 6 ? v.z : v.w));
  return (p & 1) ? (w >> 16) : (w & 0xffffu);
}

// Knuth's TwoSum: (hi, lo) += v with the rounding error of hi + v kept in lo.
__device__ __forceinline__ void ff_add(float& hi, float& lo, float v) {
  const float s = hi + v;
  const float bb = s - hi;
  const float err = (hi - (s - bb)) + (v - bb);
  hi = s;
  lo += err;
}

template <int S, int NPAD>
__global__ void __launch_bounds__(OZ_THREADS) oz_gram_kernel(const OzTile* __restrict__ tiles, int n_tiles,
                                                             const OzJob* __restrict__ jobs, const uint4* __restrict__ T,
                                                             double* __restrict__ partial, int* err, long long polls) {
  constexpr int KCH = OZ_KB * 2 / 16;                       // 16-byte K chunks per row and plane
  constexpr int A_PLANE = 128 * OZ_KB * 2, B_PLANE = NPAD * OZ_KB * 2;
  constexpr int STAGE = S * (A_PLANE + B_PLANE);
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ uint32_t tmem_slot;
  __shared__ __align__(8) uint64_t mbar[3];
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr uint32_t NCOLS = (S * NPAD <= 128) ? 128 : ((S * NPAD <= 256) ? 256 : 512);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(oz_smem_u32(&tmem_slot)),
                 "r"(NCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int i = 0; i < 3; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(oz_smem_u32(&mbar[i])), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
    s_fail = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  uint32_t uses0 = 0u, uses1 = 0u, drains = 0u;
  // D = F32, A = B = BF16 (kind::f16), both K-major, N = NPAD, M = 128
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NPAD >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);

  for (int ti = blockIdx.x; ti < n_tiles; ti += gridDim.x) {
    const OzTile tile = tiles[ti];
    // this thread's MMA row: job slot and column
    const int slot = tile.slot;                    // 32, 64 or 128 rows per job
    const int jl = tid / slot, c = tid % slot;
    const int ji = tile.job_begin + jl;
    const bool job_ok = ji < tile.job_end;
    OzJob job;
    if (job_ok) job = jobs[ji];
    const bool col_ok = job_ok && c < job.cols;
    float hi[NPAD], lo[NPAD];
#pragma unroll
    for (int j = 0; j < NPAD; ++j) { hi[j] = 0.f; lo[j] = 0.f; }

    auto load_step = [&](int r0, int b) {
      uint8_t* As = smem + b * STAGE;
      uint8_t* Bs = As + S * A_PLANE;
      // A: row (job, c), K = the OZ_KB output rows r0 .. r0 + OZ_KB
      int mp = -1;
      if (job_ok && r0 + lane < tile.r1) mp = job.map ? __ldg(job.map + r0 + lane) : ((r0 + lane) << 1);
#pragma unroll
      for (int q = 0; q < KCH; ++q) {
        uint4 e[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int src = __shfl_sync(0xffffffffu, mp, q * 8 + i);
          uint4 v = make_uint4(0u, 0u, 0u, 0u);
          if (col_ok && src >= 0) {
            v = __ldg(T + job.a_off + (long long)(src >> 1) * job.a_ld + c);
            if (src & 1) { v.x ^= 0x80008000u; v.y ^= 0x80008000u; v.z ^= 0x80008000u; v.w ^= 0x80008000u; }
          }
          e[i] = v;
        }
#pragma unroll
        for (int p = 0; p < S; ++p) {
          uint4 o;
          o.x = oz_plane(e[0], p) | (oz_plane(e[1], p) << 16);
          o.y = oz_plane(e[2], p) | (oz_plane(e[3], p) << 16);
          o.z = oz_plane(e[4], p) | (oz_plane(e[5], p) << 16);
          o.w = oz_plane(e[6], p) | (oz_plane(e[7], p) << 16);
          *(uint4*)(As + p * A_PLANE + oz_core_off(tid, q, KCH)) = o;
        }
      }
      // B: row c' of T_oc, K = rows r0 + 8 w .. + 8 (warp w), lanes over c'
#pragma unroll
      for (int cc = lane; cc < NPAD; cc += 32) {
        uint4 e[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int r = r0 + warp * 8 + i;
          e[i] = (cc < tile.n && r < tile.r1) ? __ldg(T + tile.b_off + (long long)r * tile.b_ld + cc)
                                              : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int p = 0; p < S; ++p) {
          uint4 o;
          o.x = oz_plane(e[0], p) | (oz_plane(e[1], p) << 16);
          o.y = oz_plane(e[2], p) | (oz_plane(e[3], p) << 16);
          o.z = oz_plane(e[4], p) | (oz_plane(e[5], p) << 16);
          o.w = oz_plane(e[6], p) | (oz_plane(e[7], p) << 16);
          *(uint4*)(Bs + p * B_PLANE + oz_core_off(cc, warp, KCH)) = o;
        }
      }
    };
    auto free_stage = [&](int st) {
      const uint32_t u = st ? uses1 : uses0;
      if (u > 0 && !oz_wait(oz_smem_u32(&mbar[st]), (u - 1) & 1, polls)) s_fail = 1;
    };
    // drain the MMAs so far and add the level accumulators into (hi, lo)
    auto flush = [&]() {
      if (tid == 0)
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            oz_smem_u32(&mbar[2])));
      if (!oz_wait(oz_smem_u32(&mbar[2]), drains & 1u, polls)) {
        s_fail = 1;
        oz_wait(oz_smem_u32(&mbar[2]), drains & 1u, kOzWaitPolls);
      }
      ++drains;
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
      for (int l = 0; l < S; ++l)
#pragma unroll
        for (int c0 = 0; c0 < NPAD; c0 += 16) {
          uint32_t v[16];
          const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(l * NPAD + c0);
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
              : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
              : "r"(taddr));
          asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
          for (int j = 0; j < 16; ++j) ff_add(hi[c0 + j], lo[c0 + j], __uint_as_float(v[j]));
        }
      // every thread's TMEM reads precede the next MMAs
      asm volatile("tcgen05.fence::before_thread_sync;");
    };

    const int steps = (tile.r1 - tile.r0 + OZ_KB - 1) / OZ_KB;
    int b = (int)((uses0 + uses1) & 1u);
    free_stage(b);
    load_step(tile.r0, b);
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    for (int st = 0; st < steps; ++st) {
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t a0 = oz_smem_u32(smem + b * STAGE);
        const uint32_t b0 = a0 + S * A_PLANE;
        constexpr uint32_t sbo = (uint32_t)KCH * 128u;
        const bool slab_first = (st % OZ_SLAB) == 0;
        // levels: pairs (p, q), p + q = l <= S - 1, into accumulator l
#pragma unroll
        for (int p = 0; p < S; ++p)
#pragma unroll
          for (int q = 0; q + p < S; ++q) {
            const int l = p + q;
            const uint32_t tacc = tmem + (uint32_t)(l * NPAD);
#pragma unroll
            for (int ks = 0; ks < KCH / 2; ++ks) {
              // the first product of each level in a slab overwrites it
              const uint32_t acc = (!slab_first || ks > 0 || p > 0) ? 1u : 0u;
              const uint64_t ad = oz_desc(a0 + p * A_PLANE + ks * 256, 128, sbo);
              const uint64_t bd = oz_desc(b0 + q * B_PLANE + ks * 256, 128, sbo);
              asm volatile(
                  "{\n.reg .pred pp;\nsetp.ne.b32 pp, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, pp;\n}" ::"r"(
                      tacc),
                  "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
            }
          }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            oz_smem_u32(&mbar[b])));
      }
      if (b) ++uses1; else ++uses0;
      const bool more = st + 1 < steps;
      if (more) {
        free_stage(b ^ 1);
        load_step(tile.r0 + (st + 1) * OZ_KB, b ^ 1);
      }
      if ((st % OZ_SLAB) == OZ_SLAB - 1 || !more) flush();
      asm volatile("fence.proxy.async.shared::cta;");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;");
      b ^= 1;
    }
    // FP64 partial block of this job and K range: [c][c'] at the job's slot
    if (col_ok) {
      double* dst = partial + job.part_off + (long long)tile.part * job.cols * tile.n + (long long)c * tile.n;
#pragma unroll
      for (int j = 0; j < NPAD; ++j)
        if (j < tile.n) dst[j] = (double)hi[j] + (double)lo[j];
    }
  }
  if (s_fail && tid == 0) atomicExch(err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOLS));
}

// O[c', c] (+)= sum over the output's entries (partial block, alpha) in order.
__global__ void oz_reduce_kernel(const OzOut* __restrict__ outs, const OzSum* __restrict__ sums,
                                 const double* __restrict__ partial) {
  const OzOut o = outs[blockIdx.x];
  const int mn = o.rows * o.cols;
  for (int e = threadIdx.x; e < mn; e += blockDim.x) {
    const int cp = e / o.cols, cc = e % o.cols;   // O row c' (output sector), column c (source sector)
    double s = 0.0;
    for (int k = o.sum_begin; k < o.sum_end; ++k) {
      const OzSum t = sums[k];
      double v = 0.0;
      for (int p = 0; p < t.n_parts; ++p) v += partial[t.off + (long long)p * t.part_stride + (long long)cc * o.rows + cp];
      s += t.alpha * v;
    }
    double* dst = o.O + (long long)cp * o.ld + cc;
    *dst += s;
  }
}

}  // namespace

void launch_oz_slice(const double* x, long long n, double* amax, void* planes, cudaStream_t s) {
  if (n <= 0) return;
  cudaMemsetAsync(amax, 0, sizeof(double), s);
  const int grid = (int)std::min<long long>(1216, (n + 255) / 256);
  oz_amax_kernel<<<grid, 256, 0, s>>>(x, n, amax);
  oz_slice_kernel<kOzDigits><<<grid, 256, 0, s>>>(x, n, amax, (uint4*)planes);
  count_launches(2);
}

int launch_oz_gram(const OzTile* tiles, int n_tiles, const OzJob* jobs, const void* planes, int npad, double* partial,
                   const OzOut* outs, int n_outs, const OzSum* sums, int* err, cudaStream_t s, long long polls) {
  if (n_tiles <= 0) return 0;
  if (polls < 0) polls = kOzWaitPolls;
  if (npad != 32 && npad != 64) return -7;
  constexpr int S = kOzDigits;
  const int smem = 2 * S * (128 * OZ_KB * 2 + npad * OZ_KB * 2);
  auto kern = npad == 32 ? oz_gram_kernel<S, 32> : oz_gram_kernel<S, 64>;
  static bool attr[2] = {false, false};
  if (!attr[npad == 64]) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    attr[npad == 64] = true;
  }
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  const int ncols = (S * npad <= 128) ? 128 : ((S * npad <= 256) ? 256 : 512);
  const int per_sm = std::max(1, std::min(512 / ncols, (227 * 1024) / (smem + 2048)));
  const int grid = std::min(n_tiles, sms * per_sm);
  kern<<<grid, OZ_THREADS, smem, s>>>(tiles, n_tiles, jobs, (const uint4*)planes, partial, err, polls);
  count_launches(1);
  if (n_outs > 0) {
    oz_reduce_kernel<<<n_outs, 256, 0, s>>>(outs, sums, partial);
    count_launches(1);
  }
  return 0;
}

}  // namespace qed
