// Mixed-precision H_eff x for bottom TTN nodes on the sm_103a tensor cores.
//
// y[r, :] = sum_chunks s_c(r) X_c[map_c(r), :] W_c^T  +  sum_adds alpha val(r) X32[map(r), :]
//
// The physical legs of a bottom node carry monomial site operators
// (Eq. (15) and the plaquette factors: at most one +-1 per row), so each
// product term becomes a row gather of the node tensor followed by one
// dense contraction with the environment operator on the parent leg.  The
// gather feeds the A operand of tcgen05.mma directly: every thread copies
// one gathered row into the no-swizzle K-major shared-memory layout (8-row
// x 16-byte core matrices), the environment block is the B operand, and
// all product terms of an output tile accumulate in one TMEM accumulator.
// Terms without an environment factor (site energies, the internal link of
// the pair, the constant) are added in FP64 in the epilogue.
//
// One CTA = one 128-row tile of one output charge sector; 128 threads; two
// shared-memory stages so the gather of term j+1 overlaps the MMAs of term
// j.  Every mbarrier wait is bounded (polls, a launch argument); a timeout
// sets *err, and the CTA then drains its MMAs through a commit to a fresh
// barrier (waited on with the default bound, so the MMAs still in flight
// finish before TMEM is read or freed), frees its TMEM and returns.
#include <algorithm>
#include <cuda_bf16.h>

#include <cstdio>

#include "kernels.cuh"

namespace qed {

namespace {

constexpr int TC_THREADS = 128;
constexpr long long kWaitPolls = 1LL << 22;   // default bound of one mbarrier wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, leading-dimension byte
// offset (K-direction core-matrix stride), stride-dimension byte offset
// (8-row group stride), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// byte offset of 16-byte chunk q of row r in a K-major no-swizzle tile
__device__ __forceinline__ uint32_t core_off(int r, int q, int kchunks) {
  return (uint32_t)(((r >> 3) * kchunks + q) * 128 + (r & 7) * 16);
}

__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity, long long polls = kWaitPolls) {
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

template <int ELEM>
__device__ __forceinline__ void mma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  if (ELEM == 4)
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
  else
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

template <int ELEM, bool SPLIT>
__global__ void __launch_bounds__(TC_THREADS) tc_heff_kernel(const TcTile* __restrict__ tiles,
                                                              const TcOutput* __restrict__ outs,
                                                              const TcChunk* __restrict__ chunks,
                                                              const TcAdd* __restrict__ adds, int a_bytes,
                                                              int b_bytes, int* err, long long polls) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ uint32_t tmem_slot;
  __shared__ __align__(8) uint64_t mbar[3];   // two stages, one drain
  __shared__ int s_fail;
  const TcTile tile = tiles[blockIdx.x];
  const TcOutput out = outs[tile.out];
  const int tid = threadIdx.x, warp = tid >> 5;
  uint8_t* Abuf[2] = {smem, smem + a_bytes};
  uint8_t* Bbuf[2] = {smem + 2 * a_bytes, smem + 2 * a_bytes + b_bytes};
  uint32_t ncols = 32;
  while ((int)ncols < out.npad) ncols <<= 1;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[0])), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[1])), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[2])), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
    s_fail = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  const int row = tile.row0 + tid;
  const bool row_ok = row < out.rows;
  const int nchunks = out.chunk_end - out.chunk_begin;
  // idesc: D = F32, A/B = BF16 (kind::f16) or TF32 (kind::tf32), both K-major, M = 128
  uint32_t idesc = (1u << 4) | ((uint32_t)(out.npad >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
  idesc |= ELEM == 4 ? ((2u << 7) | (2u << 10)) : ((1u << 7) | (1u << 10));

  auto load_chunk = [&](int ci, int b) {
    const TcChunk c = chunks[ci];
    const int kchunks = c.kpad * ELEM / 16;   // split: [hi | lo] for both A and B
    int src = -1;
    if (row_ok) src = c.map ? c.map[row] : (row << 1);
    const uint8_t* xrow = src >= 0 ? (const uint8_t*)c.X + (long long)(src >> 1) * c.xstride * ELEM : nullptr;
    const uint32_t flip = (src >= 0 && (src & 1)) ? (ELEM == 2 ? 0x80008000u : 0x80000000u) : 0u;
    for (int q = 0; q < kchunks; ++q) {
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (xrow) {
        v = __ldg((const uint4*)(xrow + q * 16));
        v.x ^= flip;
        v.y ^= flip;
        v.z ^= flip;
        v.w ^= flip;
      }
      *(uint4*)(Abuf[b] + core_off(tid, q, kchunks)) = v;
    }
    const uint8_t* w = (const uint8_t*)c.W;
    for (int e = tid; e < out.npad * kchunks; e += TC_THREADS) {
      const int n = e / kchunks, q = e - n * kchunks;
      *(uint4*)(Bbuf[b] + core_off(n, q, kchunks)) = __ldg((const uint4*)(w + ((long long)n * kchunks + q) * 16));
    }
  };

  uint32_t uses[2] = {0u, 0u};
  if (nchunks > 0) {
    load_chunk(out.chunk_begin, 0);
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    for (int j = 0; j < nchunks; ++j) {
      const int b = j & 1;
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        const int kchunks = chunks[out.chunk_begin + j].kpad * ELEM / 16;
        const uint32_t a0 = smem_u32(Abuf[b]), b0 = smem_u32(Bbuf[b]);
        const uint32_t sbo = (uint32_t)kchunks * 128u;
        if (!SPLIT) {
          for (int ks = 0; ks < kchunks / 2; ++ks) {
            const uint64_t ad = smem_desc(a0 + ks * 256, 128, sbo);
            const uint64_t bd = smem_desc(b0 + ks * 256, 128, sbo);
            mma<ELEM>(tmem, ad, bd, idesc, (j > 0 || ks > 0) ? 1u : 0u);
          }
        } else {
          // x_hi W_hi + x_hi W_lo + x_lo W_hi; A and B tiles hold [hi | lo]
          const int part = kchunks / 2;
          const int pa[3] = {0, 0, part}, pb[3] = {0, part, 0};
          for (int g = 0; g < 3; ++g)
            for (int ks = 0; ks < part / 2; ++ks) {
              const uint64_t ad = smem_desc(a0 + (pa[g] + 2 * ks) * 128, 128, sbo);
              const uint64_t bd = smem_desc(b0 + (pb[g] + 2 * ks) * 128, 128, sbo);
              mma<ELEM>(tmem, ad, bd, idesc, (j > 0 || g > 0 || ks > 0) ? 1u : 0u);
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&mbar[b])));
      }
      uses[b] += 1;
      if (j + 1 < nchunks) {
        const int nb = b ^ 1;
        if (uses[nb] > 0 && !mbar_wait(smem_u32(&mbar[nb]), (uses[nb] - 1) & 1, polls)) s_fail = 1;
        load_chunk(out.chunk_begin + j + 1, nb);
        asm volatile("fence.proxy.async.shared::cta;");
        __syncthreads();
      }
    }
    // drain: one more commit from the issuing thread arrives on mbar[2] once
    // every MMA it issued has completed (whatever happened to the stage
    // barriers); the wait uses the caller's bound, and after a timeout the
    // default bound, so TMEM is read and freed only after the MMAs are done
    if (tid == 0)
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&mbar[2])));
    if (!mbar_wait(smem_u32(&mbar[2]), 0, polls)) {
      s_fail = 1;
      mbar_wait(smem_u32(&mbar[2]), 0);
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
  }
  __syncthreads();
  const bool ok = s_fail == 0;
  if (!ok && tid == 0) atomicExch(err, 1);
  // epilogue: TMEM lanes 32*warp .. +31 hold rows row0 + 32*warp + lane
  for (int c0 = 0; c0 < out.n; c0 += 16) {
    uint32_t v[16];
    if (nchunks > 0) {
      const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
    } else {
      for (int j = 0; j < 16; ++j) v[j] = 0u;
    }
    if (!row_ok) continue;
    double acc[16];
    for (int j = 0; j < 16; ++j) acc[j] = ok ? (double)__uint_as_float(v[j]) : 0.0;
    for (int ai = out.add_begin; ai < out.add_end; ++ai) {
      const TcAdd a = adds[ai];
      const int src = a.map ? a.map[row] : (row << 1);
      if (src < 0) continue;
      double s = (src & 1) ? -a.alpha : a.alpha;
      if (a.val) s *= a.val[row];
      const float* xr = a.X32 + (long long)(src >> 1) * a.ld + c0;
      for (int j = 0; j < 16; ++j)
        if (c0 + j < out.n) acc[j] += s * (double)xr[j];
    }
    double* yr = out.y + (long long)row * out.n + c0;
    for (int j = 0; j < 16; ++j)
      if (c0 + j < out.n) yr[j] = acc[j];
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// One warp per padded row, lanes along the row: coalesced reads of the
// FP64 source and writes of the staged operand (no index division).
template <int ELEM, int MODE>
__global__ void __launch_bounds__(256) convert_kernel(const ConvJob* __restrict__ jobs) {
  const ConvJob j = jobs[blockIdx.y];
  const int lane = threadIdx.x & 31;
  const int warps = (int)(gridDim.x * (blockDim.x >> 5));
  for (int r = (int)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)); r < j.rows; r += warps) {
    const double* src = j.src + (long long)r * j.ld_src;
    for (int c = lane; c < j.kpad; c += 32) {
      const double v = c < j.cols ? j.scale * src[(long long)c * j.cs_src] : 0.0;
      const long long e = (long long)r * j.kpad + c;
      if (MODE == 0) {
        if (ELEM == 2)
          ((__nv_bfloat16*)j.dst)[e] = __double2bfloat16(v);
        else
          ((float*)j.dst)[e] = (float)v;
      } else {
        // [hi | lo] rows: hi = TF32-truncated, lo = FP32 residual
        const float hi = tf32_hi((float)v);
        const float lo = (float)(v - (double)hi);
        float* d = (float*)j.dst + (long long)r * 2 * j.kpad;
        d[c] = hi;
        d[j.kpad + c] = lo;
      }
      if (j.dst32) j.dst32[e] = (float)v;
    }
  }
}

}  // namespace

int launch_tc_heff(int elem, int split, const TcTile* tiles, int n_tiles, const TcOutput* outs,
                   const TcChunk* chunks, const TcAdd* adds, int max_kpad, int max_npad, int* err, cudaStream_t s,
                   long long polls) {
  if (n_tiles <= 0) return 0;
  if (polls < 0) polls = kWaitPolls;
  const int a_bytes = 128 * max_kpad * elem;
  const int b_bytes = max_npad * max_kpad * elem;
  const int smem = 2 * (a_bytes + b_bytes);
  if (smem > 200 * 1024 || max_npad > 256 || max_npad % 16 || max_kpad % 16) return -7;
  if (split && elem != 4) return -7;
  if (elem == 2) {
    static bool attr_2f = false;   // set once: host attribute calls cost as much as a launch
    if (!attr_2f) {
      cudaFuncSetAttribute(tc_heff_kernel<2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      attr_2f = true;
    }
    tc_heff_kernel<2, false><<<n_tiles, TC_THREADS, smem, s>>>(tiles, outs, chunks, adds, a_bytes, b_bytes, err, polls);
    count_launches(1);
  } else if (!split) {
    static bool attr_4f = false;   // set once: host attribute calls cost as much as a launch
    if (!attr_4f) {
      cudaFuncSetAttribute(tc_heff_kernel<4, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      attr_4f = true;
    }
    tc_heff_kernel<4, false><<<n_tiles, TC_THREADS, smem, s>>>(tiles, outs, chunks, adds, a_bytes, b_bytes, err, polls);
    count_launches(1);
  } else {
    static bool attr_4t = false;   // set once: host attribute calls cost as much as a launch
    if (!attr_4t) {
      cudaFuncSetAttribute(tc_heff_kernel<4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      attr_4t = true;
    }
    tc_heff_kernel<4, true><<<n_tiles, TC_THREADS, smem, s>>>(tiles, outs, chunks, adds, a_bytes, b_bytes, err, polls);
    count_launches(1);
  }
  return 0;
}

void launch_convert(int elem, int mode, const ConvJob* jobs, int n_jobs, long long max_elems, cudaStream_t s) {
  if (n_jobs <= 0) return;
  // rows <= max_elems / 16 (kpad >= 16); 8 rows per block, about 4 blocks per SM in total
  long long gx = (max_elems / 16 + 7) / 8;
  const long long cap = std::max(1LL, 608LL / n_jobs);
  if (gx > cap) gx = cap;
  if (gx < 1) gx = 1;
  dim3 grid((unsigned)gx, (unsigned)n_jobs);
  if (mode == 1)
    convert_kernel<4, 1><<<grid, 256, 0, s>>>(jobs);
  else if (mode == 2)
    convert_kernel<4, 2><<<grid, 256, 0, s>>>(jobs);
  else if (elem == 2)
    convert_kernel<2, 0><<<grid, 256, 0, s>>>(jobs);
  else
    convert_kernel<4, 0><<<grid, 256, 0, s>>>(jobs);
  count_launches(1);
}

}  // namespace qed
