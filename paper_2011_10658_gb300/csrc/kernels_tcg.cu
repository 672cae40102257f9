// Grouped leg contractions on the sm_103a tensor cores (tcgen05, TMEM).
//
// Every H_eff term at an upper TTN node is a Kronecker product of dense
// renormalized operators on the node's legs (Methods, "Tensor Networks",
// step (i)); applying one operator to one U(1) block of a tensor contracts
// one leg of a (d_a x d_b x d_c) block with a (d' x d) matrix.  With the two
// other legs flattened into a row index r, that is a GEMM
//     D[r, j] = alpha * sum_k A(r, k) B(j, k),
// where A(r, k) walks the block through two row strides (the two untouched
// legs) and one K stride (the contracted leg), and D is written back through
// two row strides and one column stride, so every intermediate keeps the
// (a, b, c) element order of its block.  The last stage accumulates all
// terms of one output block in one TMEM accumulator (K-concatenation over
// terms).
//
// One CTA = 128 rows of one output (MMA M = 128, one thread per row); the
// MMA N is the output width rounded up to 16.  A rows are loaded by their
// threads (FP64 or FP32 sources, converted on the integer pipes) and written
// in the no-swizzle K-major core-matrix layout; B is the operator block,
// scaled by alpha.  Two shared-memory stages: the loads of step s+1 overlap
// the MMAs of step s.  TF32 operands, optionally split (x = hi + lo, three
// products hi*hi + hi*lo + lo*hi), or BF16; FP32 accumulation.  Outputs
// whose K is long are split into parts whose FP32 partial sums are added in
// a fixed order afterwards.
//
// Every mbarrier wait is bounded (polls, a launch argument); a timeout sets
// *err, and the CTA then drains its MMAs through a commit to a fresh barrier
// (waited on with the default bound), frees its TMEM and returns.
#include <algorithm>
#include <map>

#include <cuda_bf16.h>

#include "kernels.cuh"

namespace qed {

namespace {

constexpr int TG_THREADS = 128;
constexpr int TG_KB = 16;                         // K elements per stage
constexpr long long kTgWaitPolls = 1LL << 22;

__device__ __forceinline__ uint32_t tg_smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t tg_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// byte offset of 16-byte chunk q of row r in a K-major no-swizzle tile
__device__ __forceinline__ uint32_t tg_core_off(int r, int q, int kchunks) {
  return (uint32_t)(((r >> 3) * kchunks + q) * 128 + (r & 7) * 16);
}

__device__ __forceinline__ bool tg_wait(uint32_t addr, uint32_t parity, long long polls) {
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

// FP64 -> FP32, round to nearest even, on the integer pipes (GB300 runs FP64
// instructions, conversions included, at a small fraction of its FP32 rate).
// Magnitudes below the FP32 normal range become signed zero.
__device__ __forceinline__ float tg_d2f(double d) {
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

__device__ __forceinline__ float tg_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

template <int ELEM>
__device__ __forceinline__ void tg_mma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  if (ELEM == 4)
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
  else
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

// Write 4 consecutive K values of one row into a stage: TF32 (plain or
// [hi | lo]) or BF16.  q4 = index of the group of 4 along K.
template <int ELEM, bool SPLIT>
__device__ __forceinline__ void tg_put4(uint8_t* base, int row, int q4, const float v[4]) {
  if (ELEM == 4) {
    constexpr int kch = SPLIT ? 2 * TG_KB / 4 : TG_KB / 4;
    if (SPLIT) {
      float h[4], l[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        h[i] = tg_hi(v[i]);
        l[i] = v[i] - h[i];
      }
      *(float4*)(base + tg_core_off(row, q4, kch)) = make_float4(h[0], h[1], h[2], h[3]);
      *(float4*)(base + tg_core_off(row, TG_KB / 4 + q4, kch)) = make_float4(l[0], l[1], l[2], l[3]);
    } else {
      *(float4*)(base + tg_core_off(row, q4, kch)) = make_float4(v[0], v[1], v[2], v[3]);
    }
  } else {
    // BF16: 8 elements per 16-byte chunk; q4 even / odd = low / high half
    constexpr int kch = TG_KB / 8;
    __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]);
    __nv_bfloat162 b = __floats2bfloat162_rn(v[2], v[3]);
    uint2 u;
    u.x = *(uint32_t*)&a;
    u.y = *(uint32_t*)&b;
    *(uint2*)(base + tg_core_off(row, q4 >> 1, kch) + (q4 & 1) * 8) = u;
  }
}

template <int ELEM, bool SPLIT>
__global__ void __launch_bounds__(TG_THREADS) tg_gemm_kernel(const TgTile* __restrict__ tiles, int n_tiles,
                                                              const TgOut* __restrict__ outs,
                                                              const TgChunk* __restrict__ chunks,
                                                              float* __restrict__ scratch, int a_bytes, int b_bytes,
                                                              int max_npad, int* err, long long polls) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ uint32_t tmem_slot;
  __shared__ __align__(8) uint64_t mbar[3];   // two stages, one drain
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5;
  uint32_t ncols = 32;
  while ((int)ncols < max_npad) ncols <<= 1;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tg_smem_u32(&tmem_slot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int i = 0; i < 3; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tg_smem_u32(&mbar[i])), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
    s_fail = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  // commits so far on the two stage barriers and on the drain barrier
  uint32_t uses0 = 0u, uses1 = 0u, drains = 0u;
  uint8_t* const A0 = smem;
  uint8_t* const A1 = smem + a_bytes;
  uint8_t* const B0 = smem + 2 * a_bytes;
  uint8_t* const B1 = smem + 2 * a_bytes + b_bytes;

  // stage `st` is about to be overwritten: wait for the MMAs that last read it
  auto free_stage = [&](int st) {
    const uint32_t u = st ? uses1 : uses0;
    if (u > 0 && !tg_wait(tg_smem_u32(&mbar[st]), (u - 1) & 1, polls)) s_fail = 1;
  };
  // K values k0 .. k0 + TG_KB of chunk ci of `tile` into stage buffers Ab, Bb
  auto load_step = [&](const TgTile& tile, const TgOut& out, int c_idx, int kk0, uint8_t* Ab, uint8_t* Bb) {
    const TgChunk c = chunks[c_idx];
    const int row = tile.row0 + tid;
    const bool row_ok = row < out.rows;
    long long base = 0;
    if (row_ok) base = (long long)(row / c.R2) * c.s1 + (long long)(row % c.R2) * c.s2;
#pragma unroll
    for (int q4 = 0; q4 < TG_KB / 4; ++q4) {
      float v[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int k = kk0 + 4 * q4 + i;
        float x = 0.f;
        if (row_ok && k < c.K) {
          const long long o = base + (long long)k * c.sk;
          x = c.a_f32 ? __ldg((const float*)c.A + o) : tg_d2f(__ldg((const double*)c.A + o));
        }
        v[i] = x;
      }
      tg_put4<ELEM, SPLIT>(Ab, tid, q4, v);
    }
    const float alpha = c.alpha;
    for (int e = tid; e < out.npad * (TG_KB / 4); e += TG_THREADS) {
      const int j = e / (TG_KB / 4), q4 = e % (TG_KB / 4);
      float v[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int k = kk0 + 4 * q4 + i;
        v[i] = (j < out.N && k < c.K) ? alpha * tg_d2f(__ldg(c.B + (long long)j * c.bj + (long long)k * c.bk)) : 0.f;
      }
      tg_put4<ELEM, SPLIT>(Bb, j, q4, v);
    }
  };
  // rows of `tile` from TMEM (or zeros) to the output or its partial slot
  auto store_tile = [&](const TgTile& tile, const TgOut& out, bool from_tmem, bool ok) {
    const int row = tile.row0 + tid;
    const bool row_ok = row < out.rows;
    long long cbase = 0;
    if (row_ok) cbase = (long long)(row / out.R2) * out.t1 + (long long)(row % out.R2) * out.t2;
    for (int c0 = 0; c0 < out.N; c0 += 16) {
      uint32_t v[16];
      if (from_tmem) {
        const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = 0u;
      }
      if (!row_ok) continue;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int col = c0 + j;
        if (col >= out.N) break;
        const float f = ok ? __uint_as_float(v[j]) : 0.f;
        if (tile.part >= 0) {
          scratch[out.part_off + (long long)tile.part * out.rows * out.N + (long long)row * out.N + col] = f;
        } else if (out.c_f32) {
          float* p = (float*)out.C + cbase + (long long)col * out.cj;
          *p = out.accumulate ? *p + f : f;
        } else {
          double* p = (double*)out.C + cbase + (long long)col * out.cj;
          *p = out.accumulate ? *p + (double)f : (double)f;
        }
      }
    }
  };
  // next tile of this CTA that has chunks; tiles without any get zeros
  auto next_tile = [&](int from) {
    int t = from;
    while (t < n_tiles) {
      const TgTile tl = tiles[t];
      if (tl.chunk_end > tl.chunk_begin) break;
      store_tile(tl, outs[tl.out], false, true);
      t += gridDim.x;
    }
    return t;
  };

  // The CTA walks the steps (chunk, K slab) of its tiles blockIdx.x,
  // blockIdx.x + gridDim.x, ... as one sequence on two shared-memory stages:
  // the next step's operands are loaded while the current step's MMAs run,
  // across tile boundaries too (the next tile's first step is loaded before
  // the current tile's accumulator is drained and stored).
  int ti = next_tile(blockIdx.x);
  if (ti < n_tiles) {
    TgTile tile = tiles[ti];
    TgOut out = outs[tile.out];
    int ci = tile.chunk_begin, k0 = 0, b = 0;
    bool first = true;
    load_step(tile, out, ci, k0, A0, B0);
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    while (true) {
      if (tid == 0) {
        // D = F32; A, B = TF32 (kind::tf32) or BF16 (kind::f16), K-major; M = 128
        uint32_t idesc = (1u << 4) | ((uint32_t)(out.npad >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
        idesc |= ELEM == 4 ? ((2u << 7) | (2u << 10)) : ((1u << 7) | (1u << 10));
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t a0 = tg_smem_u32(b ? A1 : A0), b0 = tg_smem_u32(b ? B1 : B0);
        if (!SPLIT) {
          constexpr int kch = TG_KB * ELEM / 16;
          constexpr uint32_t sbo = (uint32_t)kch * 128u;
#pragma unroll
          for (int ks = 0; ks < kch / 2; ++ks)
            tg_mma<ELEM>(tmem, tg_desc(a0 + ks * 256, 128, sbo), tg_desc(b0 + ks * 256, 128, sbo), idesc,
                         (!first || ks > 0) ? 1u : 0u);
        } else {
          constexpr int part = TG_KB / 4;   // 16-byte chunks of one of hi / lo
          constexpr uint32_t sbo = (uint32_t)(2 * part) * 128u;
#pragma unroll
          for (int g = 0; g < 3; ++g)
#pragma unroll
            for (int ks = 0; ks < part / 2; ++ks) {
              const int pa = g == 2 ? part : 0, pb = g == 1 ? part : 0;
              tg_mma<ELEM>(tmem, tg_desc(a0 + (pa + 2 * ks) * 128, 128, sbo),
                           tg_desc(b0 + (pb + 2 * ks) * 128, 128, sbo), idesc,
                           (!first || g > 0 || ks > 0) ? 1u : 0u);
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            tg_smem_u32(&mbar[b])));
      }
      if (b) ++uses1; else ++uses0;
      first = false;
      // the step after this one
      int nci = ci, nk0 = k0 + TG_KB, nti = ti;
      if (nk0 >= chunks[ci].K) { ++nci; nk0 = 0; }
      const bool tile_done = nci >= tile.chunk_end;
      TgTile ntile = tile;
      TgOut nout = out;
      if (tile_done) {
        nti = next_tile(ti + gridDim.x);
        if (nti < n_tiles) {
          ntile = tiles[nti];
          nout = outs[ntile.out];
          nci = ntile.chunk_begin;
          nk0 = 0;
        }
      }
      const bool more = nti < n_tiles;
      if (more) {
        free_stage(b ^ 1);
        load_step(ntile, nout, nci, nk0, b ? A0 : A1, b ? B0 : B1);
      }
      if (tile_done) {
        // drain every MMA of this tile, then its accumulator to global memory
        if (tid == 0)
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              tg_smem_u32(&mbar[2])));
        if (!tg_wait(tg_smem_u32(&mbar[2]), drains & 1u, polls)) {
          s_fail = 1;
          tg_wait(tg_smem_u32(&mbar[2]), drains & 1u, kTgWaitPolls);
        }
        ++drains;
        asm volatile("tcgen05.fence::after_thread_sync;");
        store_tile(tile, out, true, s_fail == 0);
        first = true;
      }
      if (!more) break;
      // the next step's operands are visible to the tensor cores, and every
      // TMEM read of a finished tile precedes the next tile's MMAs
      asm volatile("tcgen05.fence::before_thread_sync;");
      asm volatile("fence.proxy.async.shared::cta;");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;");
      tile = ntile;
      out = nout;
      ti = nti;
      ci = nci;
      k0 = nk0;
      b ^= 1;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (s_fail && tid == 0) atomicExch(err, 1);
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

// Partial sums of split outputs, added in part order.
__global__ void tg_reduce_kernel(const TgOut* __restrict__ outs, const int* __restrict__ red_list,
                                 const float* __restrict__ scratch) {
  const TgOut out = outs[red_list[blockIdx.y]];
  const long long mn = (long long)out.rows * out.N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < mn; e += (long long)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int p = 0; p < out.n_parts; ++p) s += scratch[out.part_off + p * mn + e];
    const int r = (int)(e / out.N), col = (int)(e % out.N);
    const long long o = (long long)(r / out.R2) * out.t1 + (long long)(r % out.R2) * out.t2 + (long long)col * out.cj;
    if (out.c_f32) {
      float* p = (float*)out.C + o;
      *p = out.accumulate ? *p + s : s;
    } else {
      double* p = (double*)out.C + o;
      *p = out.accumulate ? *p + (double)s : (double)s;
    }
  }
}

}  // namespace

int tg_stage_bytes(int elem, int split, int max_npad, int* a_bytes, int* b_bytes) {
  const int w = split ? 2 : 1;
  *a_bytes = 128 * TG_KB * elem * w;
  *b_bytes = max_npad * TG_KB * elem * w;
  return 2 * (*a_bytes + *b_bytes);
}

int launch_tg_gemm(int elem, int split, const TgTile* tiles, int n_tiles, const TgOut* outs, const TgChunk* chunks,
                   int max_npad, float* scratch, const int* red_list, int n_red, int* err, cudaStream_t s,
                   long long polls) {
  if (n_tiles <= 0) return 0;
  if (polls < 0) polls = kTgWaitPolls;
  if (max_npad > 256 || max_npad % 16 || (split && elem != 4)) return -7;
  int a_bytes = 0, b_bytes = 0;
  const int smem = tg_stage_bytes(elem, split, max_npad, &a_bytes, &b_bytes);
  if (smem > 200 * 1024) return -7;
  // kernel attributes and occupancy are looked up once per configuration
  // (host API calls of this kind cost as much as a small launch)
  const int kind = elem == 2 ? 0 : (split ? 2 : 1);
  auto kern = kind == 0 ? tg_gemm_kernel<2, false> : (kind == 2 ? tg_gemm_kernel<4, true> : tg_gemm_kernel<4, false>);
  static bool attr_set[3] = {false, false, false};
  static int sms = 0;
  if (!attr_set[kind]) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set[kind] = true;
  }
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  int ncols = 32;
  while (ncols < max_npad) ncols <<= 1;
  // CTAs per SM from the resources one CTA holds: dynamic + static shared
  // memory (227 KB per SM), TMEM columns (512 per SM), at most 8
  const int per_sm = std::max(1, std::min(8, std::min(512 / ncols, (227 * 1024) / (smem + 2048))));
  const int grid = std::min(n_tiles, sms * per_sm);
  kern<<<grid, TG_THREADS, smem, s>>>(tiles, n_tiles, outs, chunks, scratch, a_bytes, b_bytes, max_npad, err, polls);
  count_launches(1);
  if (n_red > 0) {
    tg_reduce_kernel<<<dim3(16, n_red), 256, 0, s>>>(outs, red_list, scratch);
    count_launches(1);
  }
  return 0;
}

}  // namespace qed
