// TTN sweep engine (host orchestration of the device kernels).
//
// Method (Methods, "Tensor Networks"): single-tensor optimisation with
// (i) H_eff from the Hamiltonian contracted with all other tensors,
// (ii) its lowest eigenpair by a Krylov method, (iii) the tensor replaced by
// the eigenvector, sweeping from the lowest to the highest layer.  Global
// U(1) charge conservation is built into the block structure of every
// tensor.  All other tensors are kept isometric towards the centre; a move
// of the centre is a per-sector QR (CholeskyQR2 here) whose R factor is
// absorbed by the neighbour.
#include "engine.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <stdexcept>
#include <set>

namespace qed {

namespace {
constexpr long long kKPart = 4096;     // split-K granularity for tall contractions
constexpr double kReorthRatio = 0.5;   // second Gram-Schmidt pass if ||w||^2 dropped below half
constexpr int kThickKeep = 8;          // Ritz vectors kept by a thick restart
// Centre-move QR rank handling: a sector whose QR diagonal falls below
// kQrFallback x (largest column norm) is factorised by Gram-Schmidt, where a
// remainder below kQrDependent x (largest column norm) marks a dependent
// column completed by the first unit vector with remainder above kQrAccept.
constexpr double kQrFallback = 1e-6;
constexpr double kQrDependent = 1e-9;
constexpr double kQrAccept = 0.5;
constexpr long long kZPoolBudget = 64LL << 20;   // doubles in the Z work pool for operator updates
constexpr int kOzAmax = 4000;                    // device scalar slot: max |T| of a digit-plane split
}  // namespace

// ------------------------------------------------------------------ Layout
void Layout::build(const Sectors& a, const Sectors& b, const Sectors& c, int shift_) {
  leg[0] = a;
  leg[1] = b;
  leg[2] = c;
  shift = shift_;
  blk.clear();
  index.clear();
  sec_off.assign(c.q.size(), 0);
  sec_rows.assign(c.q.size(), 0);
  long long off = 0;
  for (size_t ic = 0; ic < c.q.size(); ++ic) {
    sec_off[ic] = off;
    int rows = 0;
    for (size_t ia = 0; ia < a.q.size(); ++ia) {
      int qb = c.q[ic] + shift - a.q[ia];
      int ib = b.find(qb);
      if (ib < 0) continue;
      Blk k;
      k.ia = (int)ia;
      k.ib = ib;
      k.ic = (int)ic;
      k.da = a.dim[ia];
      k.db = b.dim[ib];
      k.dc = c.dim[ic];
      k.off = off;
      k.row0 = rows;
      index[{k.ia, k.ib}] = (int)blk.size();
      blk.push_back(k);
      off += (long long)k.da * k.db * k.dc;
      rows += k.da * k.db;
    }
    sec_rows[ic] = rows;
  }
  size = off;
}

// QED_FAIL_ALLOC_AFTER=n (read once per process): the allocation after the
// first n succeeds as if cudaMalloc had run out of memory.  A host-side fake
// of the failing call for tests of the QED_ENOMEM path.
static long long fail_alloc_after() {
  static const long long n = [] {
    const char* v = std::getenv("QED_FAIL_ALLOC_AFTER");
    return v ? std::atoll(v) : -1LL;
  }();
  return n;
}

void device_alloc(void** p, size_t bytes, const char* what) {
  *p = nullptr;
  static std::atomic<long long> count{0};
  const long long limit = fail_alloc_after();
  if (limit >= 0 && count.fetch_add(1) >= limit)
    throw DeviceAllocError(std::string(what) + ": out of memory (injected by QED_FAIL_ALLOC_AFTER)");
  const cudaError_t e = cudaMalloc(p, bytes == 0 ? 16 : bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    throw DeviceAllocError(std::string(what) + ": " + cudaGetErrorString(e));
  }
}

// ------------------------------------------------------------------ KPlan
int KPlan::add_output(double* C, long long c_m, long long c_n, int M, int N, int accumulate) {
  auto key = std::make_tuple((uintptr_t)C, c_m, c_n, M, N);
  auto it = out_index.find(key);
  if (it != out_index.end()) {
    current = it->second;
    return current;
  }
  KOutput o;
  o.C = C;
  o.c_m = c_m;
  o.c_n = c_n;
  o.M = M;
  o.N = N;
  o.chunk_begin = 0;
  o.chunk_end = 0;
  o.accumulate = accumulate;
  o.n_parts = 1;
  o.part_off = 0;
  outs.push_back(o);
  out_chunks.emplace_back();
  current = (int)outs.size() - 1;
  out_index[key] = current;
  return current;
}

void KPlan::add_chunk(const KChunk& c) { out_chunks[current].push_back(c); }

// Flatten the per-output chunk lists into the master arrays.  Tiles are cut
// per tile shape on first use (KPlan::variant).
void KPlan::finalize(long long kp) {
  if (!out_chunks.empty()) {
    chunks.clear();
    for (size_t oi = 0; oi < outs.size(); ++oi) {
      outs[oi].chunk_begin = (int)chunks.size();
      chunks.insert(chunks.end(), out_chunks[oi].begin(), out_chunks[oi].end());
      outs[oi].chunk_end = (int)chunks.size();
    }
    out_chunks.clear();
    out_index.clear();
  }
  k_part = kp;
  flops = 0.0;
  for (const KOutput& o : outs)
    for (int c = o.chunk_begin; c < o.chunk_end; ++c)
      if (!chunks[c].add) flops += 2.0 * o.M * o.N * chunks[c].K;
  for (KVariant& v : var) v.ready = false;
}

// Tiles of BM x BM (BM = 16, 32 or 64) per output.  Outputs with few tiles
// and long K are split into parts (sub-ranges of K, chunks cut where needed)
// whose partial sums go to scratch and are reduced in a fixed order
// afterwards.
KVariant& KPlan::variant(int shape, cudaStream_t s) {
  KVariant& v = var[shape];
  if (v.ready) return v;
  const int BMs = kc_shape_m(shape), BNs = kc_shape_n(shape);
  v.tiles.clear();
  v.red.clear();
  v.chunks.clear();
  v.chunks.reserve(chunks.size());
  v.outs = outs;
  v.scratch_need = 0;
  // K per part: small enough that the launch has about four tiles per SM
  // when the plan has few, long contractions (a Gram matrix), at most k_part
  long long work = 0, base_tiles = 0;
  for (const KOutput& o : outs) {
    long long ktot = 0;
    for (int c = o.chunk_begin; c < o.chunk_end; ++c) ktot += chunks[c].add ? 1 : chunks[c].K;
    const long long t = (long long)((o.M + BMs - 1) / BMs) * ((o.N + BNs - 1) / BNs);
    work += t * ktot;
    base_tiles += t;
  }
  const long long kp = std::max(256LL, std::min(k_part, work / (4 * 152)));
  const bool few_tiles = base_tiles < 4 * 152;
  std::vector<KChunk>& nc = v.chunks;
  for (size_t oi = 0; oi < outs.size(); ++oi) {
    KOutput& o = v.outs[oi];
    const KOutput& mo = outs[oi];
    const int tm = (o.M + BMs - 1) / BMs, tn = (o.N + BNs - 1) / BNs;
    long long ktot = 0;
    for (int c = mo.chunk_begin; c < mo.chunk_end; ++c) ktot += chunks[c].add ? 1 : chunks[c].K;
    const bool split = ktot > 2 * kp && (tm * tn <= 16 || few_tiles);
    std::vector<std::pair<int, int>> parts;   // ranges in nc
    const int begin = (int)nc.size();
    if (!split) {
      for (int c = mo.chunk_begin; c < mo.chunk_end; ++c) nc.push_back(chunks[c]);
      parts.push_back({begin, (int)nc.size()});
    } else {
      long long acc = 0;
      int part_begin = begin;
      for (int c = mo.chunk_begin; c < mo.chunk_end; ++c) {
        const KChunk& ch = chunks[c];
        if (ch.add) {
          nc.push_back(ch);
          acc += 1;
        } else {
          for (int k0 = 0; k0 < ch.K; k0 += (int)kp) {
            KChunk sc = ch;
            sc.K = std::min<int>((int)kp, ch.K - k0);
            if (ch.bmap) {
              sc.bmap = ch.bmap + k0;
              if (ch.bval) sc.bval = ch.bval + k0;
            } else {
              sc.B = ch.B + (long long)k0 * ch.b_k;
            }
            sc.A = ch.A + (long long)k0 * ch.a_k;
            nc.push_back(sc);
            acc += sc.K;
            if (acc >= kp) {
              parts.push_back({part_begin, (int)nc.size()});
              part_begin = (int)nc.size();
              acc = 0;
            }
          }
        }
      }
      if ((int)nc.size() > part_begin) parts.push_back({part_begin, (int)nc.size()});
    }
    o.chunk_begin = begin;
    o.chunk_end = (int)nc.size();
    if (parts.size() > 1) {
      o.n_parts = (int)parts.size();
      o.part_off = v.scratch_need;
      v.scratch_need += (long long)o.n_parts * o.M * o.N;
      v.red.push_back((int)oi);
    } else {
      o.n_parts = 1;
    }
    for (size_t pi = 0; pi < parts.size(); ++pi)
      for (int i = 0; i < tm; ++i)
        for (int j = 0; j < tn; ++j) {
          KTile t;
          t.out = (int)oi;
          t.m0 = i * BMs;
          t.n0 = j * BNs;
          t.chunk_begin = parts[pi].first;
          t.chunk_end = parts[pi].second;
          t.part = parts.size() > 1 ? (int)pi : -1;
          v.tiles.push_back(t);
        }
  }
  v.upload(s);
  v.ready = true;
  return v;
}

template <typename T>
static void grow_upload(T*& dptr, size_t& cap, const std::vector<T>& host, cudaStream_t s) {
  if (host.empty()) return;
  if (host.size() > cap) {
    if (dptr) cudaFree(dptr);
    cap = host.size() + host.size() / 2 + 16;
    device_alloc((void**)&dptr, cap * sizeof(T), "plan arrays");
  }
  cudaMemcpyAsync(dptr, host.data(), host.size() * sizeof(T), cudaMemcpyHostToDevice, s);
}

void KVariant::upload(cudaStream_t s) {
  grow_upload(d_chunks, cap_chunks, chunks, s);
  grow_upload(d_outs, cap_outs, outs, s);
  grow_upload(d_tiles, cap_tiles, tiles, s);
  grow_upload(d_red, cap_red, red, s);
}

void KVariant::release() {
  if (d_chunks) cudaFree(d_chunks);
  if (d_outs) cudaFree(d_outs);
  if (d_tiles) cudaFree(d_tiles);
  if (d_red) cudaFree(d_red);
  d_chunks = nullptr;
  d_outs = nullptr;
  d_tiles = nullptr;
  d_red = nullptr;
  cap_chunks = cap_outs = cap_tiles = cap_red = 0;
  ready = false;
}

void KPlan::release() {
  for (KVariant& v : var) v.release();
  for (auto& m : tev)
    for (auto& sh : m)
      for (auto& rep : sh)
        for (cudaEvent_t& e : rep)
          if (e) { cudaEventDestroy(e); e = nullptr; }
}

void TcPlan::release() {
  void* ptrs[6] = {d_tiles, d_outs, d_chunks, d_adds, d_xjobs, d_wjobs};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  d_tiles = nullptr; d_outs = nullptr; d_chunks = nullptr; d_adds = nullptr; d_xjobs = nullptr; d_wjobs = nullptr;
  for (size_t& c : cap) c = 0;
}

void OzPlan::release() {
  void* ptrs[4] = {d_tiles, d_jobs, d_outs, d_sums};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  d_tiles = nullptr; d_jobs = nullptr; d_outs = nullptr; d_sums = nullptr;
  for (size_t& c : cap) c = 0;
}

void TgPlan::upload(cudaStream_t s) {
  grow_upload(d_tiles, cap[0], tiles, s);
  grow_upload(d_outs, cap[1], outs, s);
  grow_upload(d_chunks, cap[2], chunks, s);
  grow_upload(d_red, cap[3], red, s);
}

void TgPlan::release() {
  void* ptrs[4] = {d_tiles, d_outs, d_chunks, d_red};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  d_tiles = nullptr; d_outs = nullptr; d_chunks = nullptr; d_red = nullptr;
  for (size_t& c : cap) c = 0;
}

static KChunk make_chunk() {
  KChunk c;
  std::memset(&c, 0, sizeof(c));
  c.alpha = 1.0;
  return c;
}

// ------------------------------------------------------------------ Engine
void* Engine::dalloc(size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  device_alloc(&p, bytes, "device tensors");
  allocs_.push_back(p);
  bytes_ += (long long)bytes;
  track(p, bytes);
  return p;
}

void Engine::dfree_all(const std::vector<void*>& ptrs) {
  std::set<void*> dead;
  for (void* p : ptrs)
    if (p) dead.insert(p);
  if (dead.empty()) return;
  cudaStreamSynchronize(stream_);
  size_t w = 0;
  for (size_t i = 0; i < allocs_.size(); ++i)
    if (!dead.count(allocs_[i])) allocs_[w++] = allocs_[i];
  allocs_.resize(w);
  for (void* p : dead) {
    auto r = ranges_.find((uintptr_t)p);
    if (r != ranges_.end()) {
      bytes_ -= (long long)r->second;
      ranges_.erase(r);
    }
    cudaFree(p);
  }
}

bool Engine::check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return true;
  err_ = std::string(what) + ": " + cudaGetErrorString(e);
  return false;
}

const SiteOp* Engine::site_op(int parity, const OpKey& key) {
  const long long packed = (((long long)(parity + 1) * 16 + key.kind) * 1024 + key.a) * 1024 + key.b;
  auto it = site_ops_.find(packed);
  if (it != site_ops_.end()) return it->second;
  SiteOp* op = new SiteOp;
  build_site_op(parity, key, op);
  site_ops_[packed] = op;
  return op;
}

bool Engine::touches_sites(int term, const std::vector<char>& reg) const {
  for (auto& so : terms_[term].ops)
    if (reg[so.first]) return true;
  return false;
}

bool Engine::touches(int term, int node) const { return touches_sites(term, in_region_[node]); }

bool Engine::inside(int term, int node) const {
  for (auto& so : terms_[term].ops)
    if (!in_region_[node][so.first]) return false;
  return true;
}

bool Engine::crosses(int term, int node) const { return touches(term, node) && !inside(term, node); }

int Engine::leg_node(int node, int leg) const {
  const TreeNode& nd = nodes_[node];
  if (leg == 2) return nd.parent;
  return nd.child_kind[leg] == 1 ? nd.child[leg] : -1;
}

int Engine::leg_site(int node, int leg) const {
  const TreeNode& nd = nodes_[node];
  return (leg < 2 && nd.child_kind[leg] == 0) ? nd.child[leg] : -1;
}

const Sectors& Engine::leg_sectors(int node, int leg) const { return layout_[node].leg[leg]; }

Layout Engine::shifted(int node, int shift) const {
  Layout L;
  L.build(layout_[node].leg[0], layout_[node].leg[1], layout_[node].leg[2], shift);
  return L;
}

void Engine::ensure_scratch(long long elems) {
  if (elems <= scratch_elems_) return;
  if (scratch_) { untrack(scratch_); cudaFree(scratch_); }
  scratch_elems_ = elems + elems / 2;
  device_alloc((void**)&scratch_, scratch_elems_ * sizeof(double), "split-K scratch");
  track(scratch_, scratch_elems_ * sizeof(double));
}

void Engine::ensure_zpool(long long elems) {
  if (elems <= zpool_elems_) return;
  clear_plan_caches();   // cached plans point into the old pool
  if (zpool_) { untrack(zpool_); cudaFree(zpool_); }
  zpool_elems_ = elems + elems / 4;
  device_alloc((void**)&zpool_, zpool_elems_ * sizeof(double), "Z pool");
  track(zpool_, zpool_elems_ * sizeof(double));
}

// [p + lo_bytes, p + hi_bytes) inside one tracked allocation?
bool Engine::in_range(const void* p, long long lo_bytes, long long hi_bytes) const {
  if (in_own_range(p, lo_bytes, hi_bytes)) return true;
  for (const Engine* e : peers_)
    if (e != this && e->in_own_range(p, lo_bytes, hi_bytes)) return true;
  return false;
}

bool Engine::in_own_range(const void* p, long long lo_bytes, long long hi_bytes) const {
  const uintptr_t a = (uintptr_t)p;
  auto it = ranges_.upper_bound(a + (lo_bytes < 0 ? 0 : 0));
  if (it == ranges_.begin()) return false;
  --it;
  const long long base = (long long)it->first, size = (long long)it->second;
  const long long lo = (long long)a + lo_bytes, hi = (long long)a + hi_bytes;
  return lo >= base && hi <= base + size;
}

// Host-side check that every chunk and output of a plan stays inside a
// known device allocation (enabled by QED_VALIDATE=1).  Row-mapped operands
// are checked over their whole source sector by the row-map builder.
bool Engine::validate_plan(const KPlan& pl, const KVariant& v, const char* what) {
  for (const KOutput& o : pl.outs) {
    const long long hi = (long long)(o.M - 1) * o.c_m + (long long)(o.N - 1) * o.c_n;
    if (o.M <= 0 || o.N <= 0 || !in_range(o.C, 0, hi * 8 + 8)) {
      err_ = std::string(what) + ": output out of range";
      return false;
    }
    for (int ci = o.chunk_begin; ci < o.chunk_end; ++ci) {
      const KChunk& c = pl.chunks[ci];
      const int K = c.add ? o.N : c.K;
      if (K <= 0) { err_ = std::string(what) + ": empty chunk"; return false; }
      if (!c.amap) {
        const long long ahi = (long long)(o.M - 1) * c.a_m + (long long)(K - 1) * c.a_k;
        if (!in_range(c.A, 0, ahi * 8 + 8)) {
          err_ = std::string(what) + ": A operand out of range";
          return false;
        }
      } else if (!in_range(c.amap, 0, (long long)o.M * 4) || (c.aval && !in_range(c.aval, 0, (long long)o.M * 8))) {
        err_ = std::string(what) + ": A row map out of range";
        return false;
      }
      if (!c.add) {
        if (!c.bmap) {
          const long long bhi = (long long)(K - 1) * c.b_k + (long long)(o.N - 1) * c.b_n;
          if (!in_range(c.B, 0, bhi * 8 + 8)) {
            err_ = std::string(what) + ": B operand out of range";
            return false;
          }
        } else if (!in_range(c.bmap, 0, (long long)K * 4) || (c.bval && !in_range(c.bval, 0, (long long)K * 8))) {
          err_ = std::string(what) + ": B row map out of range";
          return false;
        }
      }
    }
  }
  for (const KTile& t : v.tiles) {
    if (t.out < 0 || t.out >= (int)v.outs.size() || t.chunk_begin < 0 || t.chunk_end > (int)v.chunks.size()) {
      err_ = std::string(what) + ": bad tile";
      return false;
    }
    if (t.part >= 0 && !in_range(scratch_, v.outs[t.out].part_off * 8,
                                 (v.outs[t.out].part_off + (long long)(t.part + 1) * v.outs[t.out].M * v.outs[t.out].N) * 8)) {
      err_ = std::string(what) + ": scratch out of range";
      return false;
    }
  }
  return true;
}

int Engine::run_plan(KPlan& pl) {
  pl.finalize(kKPart);
  return launch_kplan(pl, 0, false);
}

// Multiply-adds a tile shape executes, padding included (split parts ignored).
double KPlan::padded_work(int shape) const {
  const double BM = kc_shape_m(shape), BN = kc_shape_n(shape);
  double w = 0.0;
  for (const KOutput& o : outs) {
    double k = 0.0;
    for (int c = o.chunk_begin; c < o.chunk_end; ++c) k += chunks[c].add ? 1.0 : chunks[c].K;
    w += std::ceil(o.M / BM) * std::ceil(o.N / BN) * BM * BN * k;
  }
  return w;
}

// Tile shapes worth timing: those whose padded work is within 1.5x of the
// least, least padded first.
int KPlan::candidates(int* out) const {
  double w[KS_COUNT], best = 1e300;
  for (int sh = 0; sh < KS_COUNT; ++sh) best = std::min(best, w[sh] = padded_work(sh));
  int n = 0;
  for (int sh = 0; sh < KS_COUNT; ++sh)
    if (w[sh] <= 1.5 * best) out[n++] = sh;
  std::sort(out, out + n, [&](int x, int y) { return w[x] < w[y]; });
  return n;
}

// Launch a plan with a tile shape.  Tuned plans (cached, replayed) are the
// autotuner's subjects: after one untimed launch with the least padded
// shape, every candidate shape (padded work within 1.5x of the least) is
// launched twice under CUDA events, interleaved, and the plan keeps the shape
// with the shortest of its two times, per arithmetic (FP64 / FP32).  Every
// launch computes the full result.  QED_KC_SHAPE=16|32|64|1664|6416 forces one shape
// (the last two: 16x64 and 64x16).
int Engine::launch_kplan(KPlan& pl, int fp32, bool tune) {
  if (pl.outs.empty()) return 0;
  const int mode = fp32;   // 0 FP64, 1 FP32, 2 float-float
  int shape = forced_shape_ >= 0 ? forced_shape_ : pl.shape[mode];
  if (shape < 0 && !tune) {   // one-off plans: the least padded shape
    int cand[KS_COUNT];
    pl.candidates(cand);
    shape = cand[0];
  }
  cudaEvent_t* timed = nullptr;
  if (shape < 0) {
    int cand[KS_COUNT];
    const int nc = pl.candidates(cand);
    const int t = pl.trials[mode];
    if (nc == 1) {
      pl.shape[mode] = shape = cand[0];
    } else if (t == 0) {
      shape = cand[0];
    } else if (t <= 2 * nc) {
      const int idx = (t - 1) % nc, rep = (t - 1) / nc;
      shape = cand[idx];
      timed = pl.tev[mode][shape][rep];
    } else {
      float best = 1e30f;
      int bs = cand[0];
      for (int i = 0; i < nc; ++i) {
        const int sh = cand[i];
        for (int rep = 0; rep < 2; ++rep) {
          cudaEvent_t* e = pl.tev[mode][sh][rep];
          float ms = 0.0f;
          if (e[0] && e[1] && cudaEventSynchronize(e[1]) == cudaSuccess &&
              cudaEventElapsedTime(&ms, e[0], e[1]) == cudaSuccess && ms < best) {
            best = ms;
            bs = sh;
          }
        }
      }
      for (auto& sh : pl.tev[mode])
        for (auto& rep : sh)
          for (cudaEvent_t& e : rep)
            if (e) { cudaEventDestroy(e); e = nullptr; }
      pl.shape[mode] = shape = bs;
    }
    pl.trials[mode] = t + 1;
  }
  KVariant& v = pl.variant(shape, stream_);
  ensure_scratch(std::max<long long>(v.scratch_need, 1));
  if (validate_ && !validate_plan(pl, v, "plan")) return -1;
  if (timed) {
    for (int i = 0; i < 2; ++i)
      if (!timed[i]) cudaEventCreate(&timed[i]);
    cudaEventRecord(timed[0], stream_);
  }
  launch_kc_gemm(v.d_tiles, (int)v.tiles.size(), v.d_outs, v.d_chunks, scratch_, stream_, fp32, shape);
  launch_kc_reduce(v.d_outs, (int)v.outs.size(), v.d_red, (int)v.red.size(), scratch_, stream_);
  if (timed) cudaEventRecord(timed[1], stream_);
  return check(cudaGetLastError(), "kc_gemm launch") ? 0 : -3;
}

KPlan* Engine::cached_plan(int kind, int a, int b, int c, const std::function<void(KPlan&)>& build) {
  const auto key = std::make_tuple(kind, a, b, c);
  auto it = plan_cache_.find(key);
  if (it != plan_cache_.end()) return it->second.get();
  std::unique_ptr<KPlan> pl(new KPlan);
  build(*pl);
  pl->finalize(kKPart);
  KPlan* raw = pl.get();
  plan_cache_[key] = std::move(pl);
  return raw;
}

void Engine::cached_plans(int kind, int a, int b, int n, KPlan** out, const std::function<void(KPlan**)>& build) {
  if (plan_cache_.find(std::make_tuple(kind, a, b, 0)) == plan_cache_.end()) {
    std::unique_ptr<KPlan> pl[4];
    KPlan* raw[4];
    for (int i = 0; i < n; ++i) {
      pl[i].reset(new KPlan);
      raw[i] = pl[i].get();
    }
    build(raw);
    for (int i = 0; i < n; ++i) {
      raw[i]->finalize(kKPart);
      plan_cache_[std::make_tuple(kind, a, b, i)] = std::move(pl[i]);
    }
  }
  for (int i = 0; i < n; ++i) out[i] = plan_cache_.at(std::make_tuple(kind, a, b, i)).get();
}

int Engine::launch_plan(KPlan* pl, int fp32) {
  ops_flops_ += pl->flops;
  return launch_kplan(*pl, fp32, true);
}

void Engine::clear_plan_caches() {
  cudaStreamSynchronize(stream_);
  ++gen_;
  plan_cache_.clear();
  heff_cache_.clear();
}

void Engine::set_precision(int p) {
  clear_tc_cache();
  precision_ = p;
  mixed_tol = p == PREC_TF32X3 ? 1e-7 : (p == PREC_TF32 ? 1e-5 : 1e-4);
}

Engine::Engine(const Params& p, int chi, uint64_t seed, int precision, cudaStream_t stream)
    : p_(p), chi_(chi), seed_(seed), precision_(precision), stream_(stream) {
  lat_ = Lattice{p.Lx, p.Ly, p.Lz, p.boundary == 1};
  const char* v = std::getenv("QED_VALIDATE");
  validate_ = v && v[0] == '1';
  if (const char* ks = std::getenv("QED_KC_SHAPE")) {
    const int d = std::atoi(ks);
    forced_shape_ = d == 16 ? KS_16 : (d == 32 ? KS_32 : (d == 64 ? KS_64 : (d == 1664 ? KS_16x64 : (d == 6416 ? KS_64x16 : -1))));
  }
  build_terms(p, &terms_, &constant_);
  nodes_ = build_tree(p.Lx, p.Ly, p.Lz);
  std::string err;
  if (!sector_table(p, chi, nodes_, &bonds_, &err)) throw std::runtime_error(err);
  const int n = (int)nodes_.size();
  in_region_.assign(n, std::vector<char>(lat_.n_sites(), 0));
  layout_.resize(n);
  for (const TreeNode& nd : nodes_) {
    for (int s : nd.sites) in_region_[nd.index][s] = 1;
    Sectors legs[2];
    for (int c = 0; c < 2; ++c)
      legs[c] = nd.child_kind[c] == 0 ? physical_sectors(lat_.parity(nd.child[c])) : bonds_[nd.child[c]];
    layout_[nd.index].build(legs[0], legs[1], bonds_[nd.index], 0);
  }
  T_.assign(n, nullptr);
  for (int i = 0; i < n; ++i) {
    T_[i] = (double*)dalloc(layout_[i].size * sizeof(double));
    nmax_ = std::max(nmax_, layout_[i].size);
  }
  up_.resize(n);
  down_.resize(n);
  x_in_ = (double*)dalloc(nmax_ * sizeof(double));
  y_out_ = (double*)dalloc(nmax_ * sizeof(double));
  tmp_ = (double*)dalloc(nmax_ * sizeof(double));
  grad_a_ = (double*)dalloc(nmax_ * sizeof(double));
  grad_b_ = (double*)dalloc(nmax_ * sizeof(double));
  grad_c_ = (double*)dalloc(nmax_ * sizeof(double));
  d_scal_ = (double*)dalloc(8192 * sizeof(double));
  d_partial_ = (double*)dalloc(1216 * (kMaxKrylov + 2) * sizeof(double));
  d_err_ = (int*)dalloc(4 * sizeof(int));   // [0] tensor-core wait flag, [1] thick-restart count, [2] non-finite flag
  if (!check(cudaStreamCreateWithFlags(&aux_, cudaStreamNonBlocking), "side stream")) throw std::runtime_error(err_);
  for (int i = 0; i <= kMaxKrylov; ++i) {
    cudaEventCreateWithFlags(&ev_iter_[i], cudaEventDisableTiming);
    cudaEventCreateWithFlags(&ev_conv_[i], cudaEventDisableTiming);
  }
  ring_dev_ = (double*)dalloc(4 * (kMaxKrylov + 1) * sizeof(double));
  if (!check(cudaMallocHost(&ring_host_, 4 * (kMaxKrylov + 1) * sizeof(double)), "pinned ring"))
    throw std::runtime_error(err_);
  cudaMemsetAsync(d_err_, 0, sizeof(int), stream_);
  long long dmax = 1;
  for (const Sectors& b : bonds_) dmax = std::max<long long>(dmax, b.total());
  qr_G_ = (double*)dalloc(dmax * dmax * sizeof(double));
  qr_Rinv_ = (double*)dalloc(dmax * dmax * sizeof(double));
  qr_Racc_ = (double*)dalloc(dmax * dmax * sizeof(double));
  qr_Rtmp_ = (double*)dalloc(dmax * dmax * sizeof(double));
  move_R_ = (double*)dalloc(dmax * dmax * sizeof(double));
  mixed_tol = precision == PREC_TF32X3 ? 1e-7 : (precision == PREC_TF32 ? 1e-5 : 1e-4);
  init_tensors();
}

Engine::~Engine() {
  cudaStreamSynchronize(stream_);
  for (auto& kv : site_ops_) delete kv.second;
  work_.release();
  plan_cache_.clear();
  heff_cache_.clear();
  tc_cache_.clear();
  for (auto& kv : qr_desc_) {
    cudaFree(kv.second.off);
    cudaFree(kv.second.n);
    cudaFree(kv.second.ld);
    cudaFree(kv.second.status);
  }
  tg_cache_.clear();
  oz_cache_.clear();
  if (oz_planes_) cudaFree(oz_planes_);
  if (oz_partial_) cudaFree(oz_partial_);
  if (tg_pool_) cudaFree(tg_pool_);
  if (tg_scratch_) cudaFree(tg_scratch_);
  if (ident_) cudaFree(ident_);
  if (xstage_) cudaFree(xstage_);
  if (xstage32_) cudaFree(xstage32_);
  if (wbuf_) cudaFree(wbuf_);
  for (auto& r : ev_pending_) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (cudaEvent_t e : ev_pool_) cudaEventDestroy(e);
  if (scratch_) cudaFree(scratch_);
  if (zpool_) cudaFree(zpool_);
  if (V_) cudaFree(V_);
  if (zb_) cudaFree(zb_);
  if (aux_) {
    cudaStreamSynchronize(aux_);
    cudaStreamDestroy(aux_);
  }
  for (int i = 0; i <= kMaxKrylov; ++i) {
    if (ev_iter_[i]) cudaEventDestroy(ev_iter_[i]);
    if (ev_conv_[i]) cudaEventDestroy(ev_conv_[i]);
  }
  if (ring_host_) cudaFreeHost(ring_host_);
  for (void* p : allocs_) cudaFree(p);
}

// SplitMix64 fill in node order, then per parent sector QR (isometry towards
// the parent; the R factor is discarded), then the renormalized operators of
// every bond, bottom-up.  The centre starts at the root.
void Engine::init_tensors() {
  uint64_t pos = 0;
  for (const TreeNode& nd : nodes_) {
    launch_fill_uniform(T_[nd.index], layout_[nd.index].size, seed_, pos, stream_);
    pos += (uint64_t)layout_[nd.index].size;
  }
  for (const TreeNode& nd : nodes_) {
    if (qr_toward(nd.index, 2, nullptr) != 0) throw std::runtime_error("initial QR: " + err_);
  }
  for (const TreeNode& nd : nodes_)
    if (nd.parent >= 0 && compute_up(nd.index) != 0) throw std::runtime_error("initial operators: " + err_);
  center_ = (int)nodes_.size() - 1;
  if (!check(cudaStreamSynchronize(stream_), "init")) throw std::runtime_error(err_);
}

// ------------------------------------------------------------------ row maps
RowMap Engine::build_rowmap_sector(int node, const SiteOp* A, const SiteOp* B, int oc,
                                   const std::vector<double>* unused) {
  (void)unused;
  const Layout& L = layout_[node];
  const int sl = leg_site(node, 0), sr = leg_site(node, 1);
  const int pl = lat_.parity(sl), pr = lat_.parity(sr);
  RowMap rm;
  const int rows = L.sec_rows[oc];
  std::vector<int> map(rows, -1);
  std::vector<double> val(rows, 0.0);
  bool need_val = false;
  int src_sec = -1;
  for (const Layout::Blk& b : L.blk) {
    if (b.ic != oc) continue;
    const int a_off = L.leg[0].offset(b.ia), b_off = L.leg[1].offset(b.ib);
    for (int a = 0; a < b.da; ++a)
      for (int c = 0; c < b.db; ++c) {
        const int row = b.row0 + a * b.db + c;
        const int ag = a_off + a, bg = b_off + c;
        const int sa = A ? A->src[ag] : ag;
        const int sb = B ? B->src[bg] : bg;
        if (sa < 0 || sb < 0) continue;
        const double v = (A ? A->val[ag] : 1.0) * (B ? B->val[bg] : 1.0);
        if (v == 0.0) continue;
        const int ia2 = L.leg[0].find(site_charge(pl, sa));
        const int ib2 = L.leg[1].find(site_charge(pr, sb));
        const int k = L.find(ia2, ib2);
        if (k < 0) continue;   // source label outside the bond sectors: zero
        const Layout::Blk& sbk = L.blk[k];
        if (src_sec >= 0 && src_sec != sbk.ic) throw std::logic_error("row map spans two sectors");
        src_sec = sbk.ic;
        const int srow = sbk.row0 + (sa - L.leg[0].offset(ia2)) * sbk.db + (sb - L.leg[1].offset(ib2));
        map[row] = (srow << 1) | (v < 0 ? 1 : 0);
        val[row] = v;
        if (std::fabs(v) != 1.0) need_val = true;
      }
  }
  rm.src_sector = src_sec;
  for (int r = 0; r < rows; ++r) rm.nnz += map[r] >= 0;
  if (src_sec < 0) return rm;
  if (need_val) {
    for (int r = 0; r < rows; ++r)
      if (map[r] >= 0) map[r] &= ~1;   // sign carried by val
  }
  rm.map = (int*)dalloc(std::max(rows, 1) * sizeof(int));
  cudaMemcpyAsync(rm.map, map.data(), rows * sizeof(int), cudaMemcpyHostToDevice, stream_);
  if (need_val) {
    rm.val = (double*)dalloc(std::max(rows, 1) * sizeof(double));
    cudaMemcpyAsync(rm.val, val.data(), rows * sizeof(double), cudaMemcpyHostToDevice, stream_);
  }
  cudaStreamSynchronize(stream_);
  return rm;
}

const std::vector<RowMap>& Engine::rowmap(int node, int term) {
  auto key = std::make_pair(node, term);
  auto it = rowmaps_.find(key);
  if (it != rowmaps_.end()) return it->second;
  const int sl = leg_site(node, 0), sr = leg_site(node, 1);
  const SiteOp* A = nullptr;
  const SiteOp* B = nullptr;
  for (auto& so : terms_[term].ops) {
    if (so.first == sl) A = site_op(lat_.parity(sl), so.second);
    if (so.first == sr) B = site_op(lat_.parity(sr), so.second);
  }
  std::vector<RowMap> maps;
  for (size_t oc = 0; oc < layout_[node].leg[2].q.size(); ++oc)
    maps.push_back(build_rowmap_sector(node, A, B, (int)oc, nullptr));
  return rowmaps_[key] = maps;
}

// Inverse of a monomial row map (the transposed operator): for each row r'
// of the source sector, the output row r with map(r) = r' and the same sign
// and factor, or none.  Built on the host from the device map, cached.
const RowMap& Engine::inverse_rowmap(const RowMap& fwd, int rows_fwd, int rows_inv) {
  auto it = inv_maps_.find(fwd.map);
  if (it != inv_maps_.end()) return it->second;
  std::vector<int> m(std::max(rows_fwd, 1));
  std::vector<double> v;
  cudaMemcpyAsync(m.data(), fwd.map, rows_fwd * sizeof(int), cudaMemcpyDeviceToHost, stream_);
  if (fwd.val) {
    v.resize(std::max(rows_fwd, 1));
    cudaMemcpyAsync(v.data(), fwd.val, rows_fwd * sizeof(double), cudaMemcpyDeviceToHost, stream_);
  }
  cudaStreamSynchronize(stream_);
  std::vector<int> im(std::max(rows_inv, 1), -1);
  std::vector<double> iv(fwd.val ? std::max(rows_inv, 1) : 0, 0.0);
  long long nnz = 0;
  for (int r = 0; r < rows_fwd; ++r) {
    if (m[r] < 0) continue;
    const int src = m[r] >> 1;
    im[src] = (r << 1) | (m[r] & 1);
    if (fwd.val) iv[src] = v[r];
    ++nnz;
  }
  RowMap inv;
  inv.src_sector = -2;   // not used for inverse maps
  inv.nnz = nnz;
  inv.map = (int*)dalloc(im.size() * sizeof(int));
  cudaMemcpyAsync(inv.map, im.data(), im.size() * sizeof(int), cudaMemcpyHostToDevice, stream_);
  if (fwd.val) {
    inv.val = (double*)dalloc(iv.size() * sizeof(double));
    cudaMemcpyAsync(inv.val, iv.data(), iv.size() * sizeof(double), cudaMemcpyHostToDevice, stream_);
  }
  cudaStreamSynchronize(stream_);
  return inv_maps_[fwd.map] = inv;
}

// Diagonal site Hamiltonian (single-site terms, one class or all) on a leg.
const std::vector<RowMap>& Engine::site_ham_map(int node, int leg, int cls) {
  auto key = std::make_pair(node, -1000 - 10 * leg - (cls + 1));
  auto it = rowmaps_.find(key);
  if (it != rowmaps_.end()) return it->second;
  const int s = leg_site(node, leg);
  SiteOp diag;
  for (int r = 0; r < kLocalDim; ++r) { diag.src[r] = (int16_t)r; diag.val[r] = 0.0; }
  diag.dq = 0;
  for (const Term& t : terms_) {
    if (t.ops.size() != 1 || t.ops[0].first != s) continue;
    if (cls >= 0 && t.cls != cls) continue;
    const SiteOp* op = site_op(lat_.parity(s), t.ops[0].second);
    for (int r = 0; r < kLocalDim; ++r)
      if (op->src[r] == r) diag.val[r] += t.coef * op->val[r];
  }
  std::vector<RowMap> maps;
  for (size_t oc = 0; oc < layout_[node].leg[2].q.size(); ++oc)
    maps.push_back(build_rowmap_sector(node, leg == 0 ? &diag : nullptr, leg == 1 ? &diag : nullptr, (int)oc,
                                       nullptr));
  return rowmaps_[key] = maps;
}

// ------------------------------------------------------------------ plans
// Y = op (x)_leg X.  op[i', i] at P (row-major dimP; transposed: P[i*dimP+i']).
// Y must be zeroed by the caller where no block of X maps.
void Engine::plan_leg_apply(KPlan& pl, const Layout& LX, const double* X, const Layout& LY, double* Y, int leg,
                            const double* P, int dimP, int shiftP, bool transposed, double alpha) {
  const Sectors& S = LX.leg[leg];
  for (const Layout::Blk& b : LX.blk) {
    int ia = b.ia, ib = b.ib;
    int ic2 = b.ic;
    int src_idx = leg == 0 ? b.ia : (leg == 1 ? b.ib : b.ic);
    int dst_idx = S.find(S.q[src_idx] + shiftP);
    if (dst_idx < 0) continue;
    if (leg == 0) ia = dst_idx;
    if (leg == 1) ib = dst_idx;
    if (leg == 2) ic2 = dst_idx;
    const int k = LY.find(ia, ib);
    if (k < 0) continue;
    const Layout::Blk& yb = LY.blk[k];
    if (yb.ic != ic2) continue;
    const long long prow = S.offset(dst_idx), pcol = S.offset(src_idx);
    // op block element (i' in dst, i in src)
    const double* Pblk = transposed ? P + pcol * dimP + prow : P + prow * dimP + pcol;
    const long long p_r = transposed ? 1 : dimP, p_c = transposed ? dimP : 1;
    if (leg == 0) {
      pl.add_output(Y + yb.off, (long long)yb.db * yb.dc, 1, yb.da, yb.db * yb.dc, 0);
      KChunk c = make_chunk();
      c.A = Pblk; c.a_m = p_r; c.a_k = p_c;
      c.B = X + b.off; c.b_k = (long long)b.db * b.dc; c.b_n = 1;
      c.K = b.da; c.alpha = alpha;
      pl.add_chunk(c);
    } else if (leg == 1) {
      for (int a = 0; a < b.da; ++a) {
        pl.add_output(Y + yb.off + (long long)a * yb.db * yb.dc, yb.dc, 1, yb.db, yb.dc, 0);
        KChunk c = make_chunk();
        c.A = Pblk; c.a_m = p_r; c.a_k = p_c;
        c.B = X + b.off + (long long)a * b.db * b.dc; c.b_k = b.dc; c.b_n = 1;
        c.K = b.db; c.alpha = alpha;
        pl.add_chunk(c);
      }
    } else {
      pl.add_output(Y + yb.off, yb.dc, 1, yb.da * yb.db, yb.dc, 0);
      KChunk c = make_chunk();
      c.A = X + b.off; c.a_m = b.dc; c.a_k = 1;
      // B[k, n] = op[n, k]
      c.B = Pblk; c.b_k = p_c; c.b_n = p_r;
      c.K = b.dc; c.alpha = alpha;
      pl.add_chunk(c);
    }
  }
}

// O[i', i] (dimO x dimO, accumulated) += alpha * sum over the other two legs
// of T[.., i', ..] Z[.., i, ..], T in layout LT (shift 0), Z in LZ.
// Each output block is one output; contributions are chunks.
void Engine::plan_contract_but(KPlan& pl, const Layout& LT, const double* T, const Layout& LZ, const double* Z,
                               int leg, double* O, int dimO, double alpha) {
  const Sectors& S = LT.leg[leg];
  std::map<std::pair<int, int>, std::vector<KChunk>> acc;   // (i'-sector, i-sector) -> chunks
  if (leg == 2) {
    for (size_t ic1 = 0; ic1 < LT.sec_rows.size(); ++ic1) {
      const int rows = LT.sec_rows[ic1];
      if (rows == 0) continue;
      // Z rows with the same (a, b) blocks have label q' - shift
      const int ic = S.find(S.q[ic1] - LZ.shift);
      if (ic < 0 || LZ.sec_rows[ic] != rows) continue;
      KChunk c = make_chunk();
      c.A = T + LT.sec_off[ic1]; c.a_m = 1; c.a_k = S.dim[ic1];
      c.B = Z + LZ.sec_off[ic]; c.b_k = S.dim[ic]; c.b_n = 1;
      c.K = rows; c.alpha = alpha;
      acc[{(int)ic1, ic}].push_back(c);
    }
  } else {
    for (const Layout::Blk& tb : LT.blk) {
      // Z block with the same other-leg indices; this leg shifted by +LZ.shift
      int ia = tb.ia, ib = tb.ib;
      int idx = leg == 0 ? tb.ia : tb.ib;
      int zidx = S.find(S.q[idx] + LZ.shift);
      if (zidx < 0) continue;
      if (leg == 0) ia = zidx; else ib = zidx;
      const int k = LZ.find(ia, ib);
      if (k < 0) continue;
      const Layout::Blk& zb = LZ.blk[k];
      if (zb.ic != tb.ic) continue;
      if (leg == 0) {
        KChunk c = make_chunk();
        c.A = T + tb.off; c.a_m = (long long)tb.db * tb.dc; c.a_k = 1;
        c.B = Z + zb.off; c.b_k = 1; c.b_n = (long long)zb.db * zb.dc;
        c.K = tb.db * tb.dc; c.alpha = alpha;
        acc[{tb.ia, zb.ia}].push_back(c);
      } else {
        for (int a = 0; a < tb.da; ++a) {
          KChunk c = make_chunk();
          c.A = T + tb.off + (long long)a * tb.db * tb.dc; c.a_m = tb.dc; c.a_k = 1;
          c.B = Z + zb.off + (long long)a * zb.db * zb.dc; c.b_k = 1; c.b_n = zb.dc;
          c.K = tb.dc; c.alpha = alpha;
          acc[{tb.ib, zb.ib}].push_back(c);
        }
      }
    }
  }
  for (auto& kv : acc) {
    const int i1 = kv.first.first, i0 = kv.first.second;
    pl.add_output(O + S.offset(i1) * dimO + S.offset(i0), dimO, 1, S.dim[i1], S.dim[i0], 1);
    for (const KChunk& c : kv.second) pl.add_chunk(c);
  }
}

// ------------------------------------------------------------------ QR
enum PlanKind { PK_UP = 1, PK_DOWN = 2, PK_QR_GRAM = 3, PK_QR_APPLY = 4, PK_QR_RACC = 5, PK_ABSORB = 6 };

// CholeskyQR2 of T[node] with `leg` as the column index, per sector of that
// leg.  T <- Q.  If Rout != nullptr, R (dim x dim, block diagonal) is written.
// An ill-conditioned or rank-deficient sector sends the whole leg to the
// Gram-Schmidt fallback (qr_gram_schmidt).
int Engine::qr_toward(int node, int leg, double* Rout) {
  const Layout& L = layout_[node];
  const Sectors& S = L.leg[leg];
  const int dim = S.total();
  const long long dd = (long long)dim * dim;
  double* Gb = qr_G_;
  double* Rinv = qr_Rinv_;
  double* Racc = qr_Racc_;
  double* Rtmp = qr_Rtmp_;
  auto dit = qr_desc_.find({node, leg});
  if (dit == qr_desc_.end()) {
    std::vector<long long> off;
    std::vector<int> nn, ld;
    QrDesc d;
    for (size_t i = 0; i < S.q.size(); ++i) {
      off.push_back(S.offset((int)i) * dim + S.offset((int)i));
      nn.push_back(S.dim[i]);
      ld.push_back(dim);
      d.max_n = std::max(d.max_n, S.dim[i]);
    }
    d.count = (int)nn.size();
    device_alloc((void**)&d.off, off.size() * sizeof(long long), "QR descriptors");
    device_alloc((void**)&d.n, nn.size() * sizeof(int), "QR descriptors");
    device_alloc((void**)&d.ld, ld.size() * sizeof(int), "QR descriptors");
    device_alloc((void**)&d.status, nn.size() * sizeof(int), "QR descriptors");
    cudaMemcpyAsync(d.off, off.data(), off.size() * sizeof(long long), cudaMemcpyHostToDevice, stream_);
    cudaMemcpyAsync(d.n, nn.data(), nn.size() * sizeof(int), cudaMemcpyHostToDevice, stream_);
    cudaMemcpyAsync(d.ld, ld.data(), ld.size() * sizeof(int), cudaMemcpyHostToDevice, stream_);
    dit = qr_desc_.emplace(std::make_pair(node, leg), d).first;
  }
  const QrDesc& d = dit->second;
  if (d.max_n > 160) {
    err_ = "sector dimension above 160 is not supported by the QR kernel";
    return -7;
  }
  double* T = T_[node];
  KPlan* gram = cached_plan(PK_QR_GRAM, node, leg, 0, [&](KPlan& pl) {
    plan_contract_but(pl, L, T, L, T, leg, Gb, dim, 1.0);
  });
  KPlan* apply = cached_plan(PK_QR_APPLY, node, leg, 0, [&](KPlan& pl) {
    plan_leg_apply(pl, L, T, L, tmp_, leg, Rinv, dim, 0, true, 1.0);
  });
  KPlan* racc = cached_plan(PK_QR_RACC, node, leg, 0, [&](KPlan& pl) {
    for (size_t i = 0; i < S.q.size(); ++i) {
      const long long o = S.offset((int)i);
      pl.add_output(Rtmp + o * dim + o, dim, 1, S.dim[i], S.dim[i], 0);
      KChunk c = make_chunk();
      c.A = Gb + o * dim + o; c.a_m = dim; c.a_k = 1;
      c.B = Racc + o * dim + o; c.b_k = dim; c.b_n = 1;
      c.K = S.dim[i];
      pl.add_chunk(c);
    }
  });
  int rc = 0;
  bool fallback = false;
  for (int pass = 0; pass < 2 && rc == 0; ++pass) {
    cudaMemsetAsync(Gb, 0, dd * sizeof(double), stream_);
    rc = launch_plan(gram);
    if (rc) break;
    cudaMemsetAsync(Rinv, 0, dd * sizeof(double), stream_);
    launch_cholesky_inv(Gb, Rinv, d.off, d.n, d.ld, d.count, d.max_n, kQrFallback * kQrFallback, d.status, stream_);
    std::vector<int> status(d.count);
    cudaMemcpyAsync(status.data(), d.status, d.count * sizeof(int), cudaMemcpyDeviceToHost, stream_);
    if (!check(cudaStreamSynchronize(stream_), "cholesky")) { rc = -3; break; }
    for (int st : status)
      if (st) fallback = true;
    if (fallback) {
      if (pass == 0) break;
      // a second pass of a well-conditioned first pass cannot be ill-conditioned
      err_ = "CholeskyQR: second pass lost positive definiteness";
      rc = -5;
      break;
    }
    // T <- T (x)_leg Rinv^T  (Q = X R^{-1})
    cudaMemsetAsync(tmp_, 0, L.size * sizeof(double), stream_);
    rc = launch_plan(apply);
    if (rc) break;
    launch_copy(tmp_, T, L.size, stream_);
    // R accumulation: Racc = R_pass * Racc (R of this pass in Gb, upper)
    if (pass == 0) {
      cudaMemcpyAsync(Racc, Gb, dd * sizeof(double), cudaMemcpyDeviceToDevice, stream_);
    } else {
      cudaMemsetAsync(Rtmp, 0, dd * sizeof(double), stream_);
      rc = launch_plan(racc);
      cudaMemcpyAsync(Racc, Rtmp, dd * sizeof(double), cudaMemcpyDeviceToDevice, stream_);
    }
  }
  if (rc == 0 && fallback) rc = qr_gram_schmidt(node, leg, Racc);
  if (rc == 0 && Rout) cudaMemcpyAsync(Rout, Racc, dd * sizeof(double), cudaMemcpyDeviceToDevice, stream_);
  return rc;
}

// Rows of the sector matrices of T[node] with `leg` as the column index,
// ordered lexicographically in the two other legs.  Each view piece is
// (block, first row in its sector, rows of the piece, row stride a).
struct SectorPiece { int blk; long long row0; int a; };

// Gram-Schmidt fallback for ill-conditioned or rank-deficient sectors:
// gather every sector of `leg` into column-major workspaces, factorise, and
// scatter Q back.  R (dim x dim, block diagonal) goes to Rout.
int Engine::qr_gram_schmidt(int node, int leg, double* Rout) {
  const Layout& L = layout_[node];
  const Sectors& S = L.leg[leg];
  const int dim = S.total();
  const int ns = (int)S.q.size();
  std::vector<long long> rows(ns, 0), woff(ns, 0);
  // order of blocks: by the sector of the first remaining leg
  std::vector<std::vector<int>> blocks(ns);
  for (int bi = 0; bi < (int)L.blk.size(); ++bi) {
    const Layout::Blk& b = L.blk[bi];
    blocks[leg == 0 ? b.ia : (leg == 1 ? b.ib : b.ic)].push_back(bi);
  }
  for (int i = 0; i < ns; ++i) {
    std::sort(blocks[i].begin(), blocks[i].end(), [&](int x, int y) {
      const Layout::Blk& a = L.blk[x];
      const Layout::Blk& b = L.blk[y];
      if (leg == 0) return a.ib < b.ib;
      return a.ia < b.ia;   // leg 1: a outer; leg 2: blocks already in (q_a) order
    });
    for (int bi : blocks[i]) {
      const Layout::Blk& b = L.blk[bi];
      rows[i] += leg == 0 ? (long long)b.db * b.dc : (leg == 1 ? (long long)b.da * b.dc : (long long)b.da * b.db);
    }
    if (rows[i] < S.dim[i]) {
      err_ = "QR: a sector has fewer rows than columns";
      return -7;
    }
  }
  long long total = 0;
  for (int i = 0; i < ns; ++i) { woff[i] = total; total += rows[i] * S.dim[i]; }
  double* W = nullptr;
  if (!check(cudaMalloc(&W, std::max(total, 1LL) * sizeof(double)), "QR workspace")) return -2;
  track(W, std::max(total, 1LL) * sizeof(double));
  double* T = T_[node];
  int rc = 0;
  for (int dir = 0; dir < 2 && rc == 0; ++dir) {   // 0 gather, 1 scatter
    work_.clear();
    for (int i = 0; i < ns; ++i) {
      long long r0 = 0;
      const long long m = rows[i];
      for (int bi : blocks[i]) {
        const Layout::Blk& b = L.blk[bi];
        double* tb = T + b.off;
        double* wb = W + woff[i] + r0;
        if (leg == 2 || leg == 0) {
          // leg 2: T block is (da*db) x dc row-major, rows in place
          // leg 0: rows (b, c) of a block are its columns (b*dc + c), cols a
          const int M = leg == 2 ? b.da * b.db : b.db * b.dc;
          const int N = leg == 2 ? b.dc : b.da;
          const long long t_m = leg == 2 ? b.dc : 1, t_n = leg == 2 ? 1 : (long long)b.db * b.dc;
          KChunk c = make_chunk();
          c.add = 1;
          if (dir == 0) {
            work_.add_output(wb, 1, m, M, N, 0);
            c.A = tb; c.a_m = t_m; c.a_k = t_n;
          } else {
            work_.add_output(tb, t_m, t_n, M, N, 0);
            c.A = wb; c.a_m = 1; c.a_k = m;
          }
          work_.add_chunk(c);
          r0 += M;
        } else {
          for (int a = 0; a < b.da; ++a) {
            // rows (a, c), c inner; cols b: T[a, b, c] at a*db*dc + b*dc + c
            KChunk c = make_chunk();
            c.add = 1;
            double* ta = tb + (long long)a * b.db * b.dc;
            if (dir == 0) {
              work_.add_output(wb + (long long)a * b.dc, 1, m, b.dc, b.db, 0);
              c.A = ta; c.a_m = 1; c.a_k = b.dc;
            } else {
              work_.add_output(ta, 1, b.dc, b.dc, b.db, 0);
              c.A = wb + (long long)a * b.dc; c.a_m = 1; c.a_k = m;
            }
            work_.add_chunk(c);
          }
          r0 += (long long)b.da * b.dc;
        }
      }
    }
    rc = run_plan(work_);
    if (rc == 0 && dir == 0) {
      std::vector<long long> roff(ns);
      std::vector<int> ri(ns), ci(ns);
      for (int i = 0; i < ns; ++i) {
        roff[i] = S.offset(i) * (long long)dim + S.offset(i);
        ri[i] = (int)rows[i];
        ci[i] = S.dim[i];
        if (ci[i] > 256) { err_ = "QR: sector dimension above 256"; rc = -7; }
      }
      if (rc) break;
      long long* d_w = nullptr;
      long long* d_r = nullptr;
      int *d_rows = nullptr, *d_cols = nullptr;
      device_alloc((void**)&d_w, ns * sizeof(long long), "QR descriptors");
      device_alloc((void**)&d_r, ns * sizeof(long long), "QR descriptors");
      device_alloc((void**)&d_rows, ns * sizeof(int), "QR descriptors");
      device_alloc((void**)&d_cols, ns * sizeof(int), "QR descriptors");
      cudaMemcpyAsync(d_w, woff.data(), ns * sizeof(long long), cudaMemcpyHostToDevice, stream_);
      cudaMemcpyAsync(d_r, roff.data(), ns * sizeof(long long), cudaMemcpyHostToDevice, stream_);
      cudaMemcpyAsync(d_rows, ri.data(), ns * sizeof(int), cudaMemcpyHostToDevice, stream_);
      cudaMemcpyAsync(d_cols, ci.data(), ns * sizeof(int), cudaMemcpyHostToDevice, stream_);
      cudaMemsetAsync(Rout, 0, (size_t)dim * dim * sizeof(double), stream_);
      launch_cgs2_qr(W, d_w, d_rows, d_cols, ns, Rout, d_r, dim, kQrDependent, kQrAccept, stream_);
      rc = check(cudaStreamSynchronize(stream_), "Gram-Schmidt QR") ? 0 : -3;
      cudaFree(d_w);
      cudaFree(d_r);
      cudaFree(d_rows);
      cudaFree(d_cols);
    }
  }
  cudaStreamSynchronize(stream_);
  untrack(W);
  cudaFree(W);
  return rc;
}

// T[node] <- R (x)_leg T[node]  (R is always the move buffer)
int Engine::absorb(int node, int leg, const double* R) {
  const Layout& L = layout_[node];
  const int dim = L.leg[leg].total();
  KPlan* pl = cached_plan(PK_ABSORB, node, leg, 0, [&](KPlan& p) {
    plan_leg_apply(p, L, T_[node], L, tmp_, leg, R, dim, 0, false, 1.0);
  });
  cudaMemsetAsync(tmp_, 0, L.size * sizeof(double), stream_);
  int rc = launch_plan(pl);
  launch_copy(tmp_, T_[node], L.size, stream_);
  return rc;
}

// ------------------------------------------------------------------ bond operators

// Renormalized operators of the bond above `node` (subtree side), from
// T[node] (isometric towards its parent) and the operators below it.
int Engine::compute_up(int node) {
  const TreeNode& nd = nodes_[node];
  const Layout& L = layout_[node];
  const int dim = L.leg[2].total();
  const long long dd = (long long)dim * dim;
  BondOps& out = up_[node];
  const bool bottom = nd.child_kind[0] == 0;
  const double* T = T_[node];
  auto op_ptr = [&](int key, int shift) -> double* {
    auto it = out.term.find(key);
    if (it == out.term.end()) {
      BondOp b;
      b.ptr = (double*)dalloc(dd * sizeof(double));
      b.shift = shift;
      it = out.term.emplace(key, b).first;
    }
    it->second.shift = shift;
    return it->second.ptr;
  };
  for (int c = 0; c < N_CLASSES; ++c)
    if (!out.H[c]) out.H[c] = (double*)dalloc(dd * sizeof(double));
  if (!out.Htot) out.Htot = (double*)dalloc(dd * sizeof(double));
  // Contributions: (output matrix, alpha, op on leg 0, op on leg 1) where an
  // op is identified by (term or site-ham), shift.
  struct Contrib { double* O; double alpha; int term; int kind; int cls; };
  // kind: 0 crossing term op, 1 term inside (coef), 2 site/child Hamiltonian of leg (term = leg)
  std::vector<Contrib> cs;
  for (int k = 0; k < (int)terms_.size(); ++k) {
    if (crosses(k, node)) {
      int d = 0;
      for (auto& so : terms_[k].ops)
        if (in_region_[node][so.first]) {
          const SiteOp* op = site_op(lat_.parity(so.first), so.second);
          d += op->dq;
        }
      cs.push_back({op_ptr(k, d), 1.0, k, 0, -1});
    } else if (inside(k, node)) {
      // inside terms touching both children (or, at the bottom, single-site terms too)
      bool tl = false, tr = false;
      for (auto& so : terms_[k].ops) {
        for (int leg = 0; leg < 2; ++leg) {
          int cn = leg_node(node, leg), cs_ = leg_site(node, leg);
          bool in = cn >= 0 ? in_region_[cn][so.first] : so.first == cs_;
          if (in) (leg == 0 ? tl : tr) = true;
        }
      }
      if (tl && tr) cs.push_back({out.H[terms_[k].cls], terms_[k].coef, k, 1, terms_[k].cls});
    }
  }
  for (int c = 0; c < N_CLASSES; ++c) cudaMemsetAsync(out.H[c], 0, dd * sizeof(double), stream_);
  for (auto& kv : out.term) cudaMemsetAsync(kv.second.ptr, 0, dd * sizeof(double), stream_);
  int rc = 0;
  int max_sector = 0;
  for (int d : L.leg[2].dim) max_sector = std::max(max_sector, d);
  if (bottom && precision_ != PREC_FP64 && max_sector <= 64) {
    // mixed states: FP64-accurate digit-plane products on the tensor cores
    // (output sectors up to 64 wide; wider ones take the FP64 kernel below)
    std::vector<std::pair<double*, double>> oc_terms;
    std::vector<int> oc_keys;
    for (const Contrib& c : cs) {
      oc_terms.push_back({c.O, c.alpha});
      oc_keys.push_back(c.term);
    }
    rc = compute_up_oz(node, oc_terms, oc_keys, out);
  } else if (bottom) {
    // term contributions through row maps: O[c', c] += alpha sum_r T[r, c'] val(r) T[map(r), c]
    KPlan* pl = cached_plan(PK_UP, node, 0, 0, [&](KPlan& w) {
      auto add_map = [&](double* O, double alpha, const std::vector<RowMap>& maps) {
        for (size_t oc = 0; oc < maps.size(); ++oc) {
          const RowMap& rm = maps[oc];
          if (rm.src_sector < 0 || L.sec_rows[oc] == 0) continue;
          const int ic = rm.src_sector;
          w.add_output(O + L.leg[2].offset((int)oc) * dim + L.leg[2].offset(ic), dim, 1, L.leg[2].dim[oc],
                       L.leg[2].dim[ic], 1);
          KChunk c = make_chunk();
          c.A = T + L.sec_off[oc]; c.a_m = 1; c.a_k = L.leg[2].dim[oc];
          c.B = T + L.sec_off[ic]; c.b_k = L.leg[2].dim[ic]; c.b_n = 1;
          c.bmap = rm.map; c.bval = rm.val;
          c.K = L.sec_rows[oc]; c.alpha = alpha;
          w.add_chunk(c);
        }
      };
      for (const Contrib& c : cs) add_map(c.O, c.alpha, rowmap(node, c.term));
      for (int leg = 0; leg < 2; ++leg)
        for (int cl = 0; cl < N_CLASSES; ++cl) add_map(out.H[cl], 1.0, site_ham_map(node, leg, cl));
    });
    rc = launch_plan(pl);
  } else {
    // upper node: Z = (A (x) B) T into pool buffers, then O += T^T Z
    struct Job { double* O; double alpha; int shA, shB; const double* A; const double* B; };
    std::vector<Job> jobs;
    for (const Contrib& c : cs) {
      Job j{c.O, c.alpha, 0, 0, nullptr, nullptr};
      for (int leg = 0; leg < 2; ++leg) {
        int cn = leg_node(node, leg);
        if (!touches(c.term, cn)) continue;
        const BondOp& bo = up_[cn].term.at(c.term);
        (leg == 0 ? j.A : j.B) = bo.ptr;
        (leg == 0 ? j.shA : j.shB) = bo.shift;
      }
      jobs.push_back(j);
    }
    for (int leg = 0; leg < 2; ++leg) {
      int cn = leg_node(node, leg);
      for (int cl = 0; cl < N_CLASSES; ++cl) {
        Job j{out.H[cl], 1.0, 0, 0, nullptr, nullptr};
        (leg == 0 ? j.A : j.B) = up_[cn].H[cl];
        jobs.push_back(j);
      }
    }
    // process in batches that fit the Z pool
    long long zsize = 0;
    for (int s = -2; s <= 2; ++s) zsize = std::max(zsize, shifted(node, s).size);
    const int batch = std::max<int>(1, (int)std::min<long long>((long long)jobs.size(), kZPoolBudget / (2 * std::max(1LL, zsize))));
    ensure_zpool(2 * batch * zsize);
    std::map<int, Layout> lays;
    for (int s = -2; s <= 2; ++s) lays[s] = shifted(node, s);
    const int dl = L.leg[0].total(), dr = L.leg[1].total();
    for (size_t j0 = 0, bi = 0; j0 < jobs.size() && rc == 0; j0 += batch, ++bi) {
      const size_t j1 = std::min(jobs.size(), j0 + batch);
      cudaMemsetAsync(zpool_, 0, 2 * batch * zsize * sizeof(double), stream_);
      KPlan* st[3];
      cached_plans(PK_UP, node, (int)bi + 1, 3, st, [&](KPlan** p) {
        for (size_t j = j0; j < j1; ++j) {
          const Job& jb = jobs[j];
          double* z1 = zpool_ + (2 * (j - j0)) * zsize;
          double* z2 = z1 + zsize;
          const double* Z = nullptr;
          int shift = 0;
          if (jb.A && jb.B) {
            plan_leg_apply(*p[0], L, T, lays[jb.shA], z1, 0, jb.A, dl, jb.shA, false, 1.0);
            plan_leg_apply(*p[1], lays[jb.shA], z1, lays[jb.shA + jb.shB], z2, 1, jb.B, dr, jb.shB, false, 1.0);
            Z = z2;
            shift = jb.shA + jb.shB;
          } else if (jb.A) {
            plan_leg_apply(*p[0], L, T, lays[jb.shA], z1, 0, jb.A, dl, jb.shA, false, 1.0);
            Z = z1;
            shift = jb.shA;
          } else {
            plan_leg_apply(*p[0], L, T, lays[jb.shB], z1, 1, jb.B, dr, jb.shB, false, 1.0);
            Z = z1;
            shift = jb.shB;
          }
          plan_contract_but(*p[2], L, T, lays[shift], Z, 2, jb.O, dim, jb.alpha);
        }
      });
      for (int i = 0; i < 3 && rc == 0; ++i) rc = launch_plan(st[i], ops_mode());
    }
  }
  // Htot = sum of classes
  cudaMemsetAsync(out.Htot, 0, dd * sizeof(double), stream_);
  for (int c = 0; c < N_CLASSES; ++c) launch_add_scaled(out.H[c], out.Htot, dd, 1.0, stream_);
  return rc;
}

// Operators of the bond above bottom node `node` on the BF16 tensor cores
// at FP64-level accuracy (digit planes, kernels_oz.cu): every term with a
// signed row map contributes O[oc-block, ic-block] += alpha T_oc^T T_ic[map];
// each site Hamiltonian of a coupling class (a diagonal row scaling) is
// split into one 0/1 row selection per distinct value v, with alpha = v.
// terms[i] / keys[i]: output operator and coefficient of term keys[i].
int Engine::compute_up_oz(int node, const std::vector<std::pair<double*, double>>& terms,
                          const std::vector<int>& keys, BondOps& out) {
  const Layout& L = layout_[node];
  const Sectors& P = L.leg[2];
  const int dim = P.total();
  const int ns = (int)P.q.size();
  if (!oz_planes_) {
    device_alloc((void**)&oz_planes_, (size_t)nmax_ * 16, "digit planes");
    track(oz_planes_, (size_t)nmax_ * 16);
  }
  auto it = oz_cache_.find(node);
  if (it == oz_cache_.end()) {
    std::unique_ptr<OzPlan> pl(new OzPlan);
    OzPlan& op = *pl;
    struct J { const int* map; int oc, ic; double* O; double alpha; long long nnz; };
    std::vector<J> js;
    for (size_t i = 0; i < terms.size(); ++i) {
      const std::vector<RowMap>& maps = rowmap(node, keys[i]);
      for (int oc = 0; oc < ns; ++oc) {
        const RowMap& rm = maps[oc];
        if (rm.src_sector < 0 || L.sec_rows[oc] == 0) continue;
        if (rm.val) { err_ = "digit-plane operator update: valued row map of a term"; return -7; }
        js.push_back({rm.map, oc, rm.src_sector, terms[i].first, terms[i].second, rm.nnz});
      }
    }
    // site Hamiltonians per leg and class: 0/1 row selections per distinct value
    const int sites[2] = {leg_site(node, 0), leg_site(node, 1)};
    for (int leg = 0; leg < 2; ++leg) {
      const int st = sites[leg];
      for (int cl = 0; cl < N_CLASSES; ++cl) {
        double diag[kLocalDim];
        for (int r = 0; r < kLocalDim; ++r) diag[r] = 0.0;
        for (const Term& t : terms_) {
          if (t.ops.size() != 1 || t.ops[0].first != st || t.cls != cl) continue;
          const SiteOp* so = site_op(lat_.parity(st), t.ops[0].second);
          for (int r = 0; r < kLocalDim; ++r)
            if (so->src[r] == r) diag[r] += t.coef * so->val[r];
        }
        std::vector<double> vals;
        for (int r = 0; r < kLocalDim; ++r)
          if (diag[r] != 0.0 && std::find(vals.begin(), vals.end(), diag[r]) == vals.end()) vals.push_back(diag[r]);
        for (double v : vals) {
          for (int oc = 0; oc < ns; ++oc) {
            const int rows = L.sec_rows[oc];
            if (rows == 0) continue;
            std::vector<int> m(rows, -1);
            long long nnz = 0;
            for (const Layout::Blk& b : L.blk) {
              if (b.ic != oc) continue;
              const int a_off = L.leg[0].offset(b.ia), b_off = L.leg[1].offset(b.ib);
              for (int a = 0; a < b.da; ++a)
                for (int c = 0; c < b.db; ++c) {
                  const int idx = leg == 0 ? a_off + a : b_off + c;
                  if (diag[idx] == v) {
                    const int r = b.row0 + a * b.db + c;
                    m[r] = r << 1;
                    ++nnz;
                  }
                }
            }
            if (!nnz) continue;
            int* dm = (int*)dalloc((size_t)rows * sizeof(int));
            op.owned.push_back(dm);
            cudaMemcpyAsync(dm, m.data(), (size_t)rows * sizeof(int), cudaMemcpyHostToDevice, stream_);
            js.push_back({dm, oc, oc, out.H[cl], v, nnz});
          }
        }
      }
    }
    cudaStreamSynchronize(stream_);
    // tiles: jobs of one output sector share the T_oc operand; up to four
    // jobs of at most 32 columns per CTA; the rows of the sector are cut
    // into K ranges (multiples of 32) so that the launch fills the GPU
    std::vector<int> order(js.size());
    for (size_t i = 0; i < js.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return js[a].oc < js[b].oc; });
    int maxd = 0;
    for (int i = 0; i < ns; ++i) maxd = std::max(maxd, P.dim[i]);
    const int slot = maxd <= 32 ? 32 : (maxd <= 64 ? 64 : 128);
    op.npad = maxd <= 32 ? 32 : 64;
    if (maxd > 64) { err_ = "digit-plane operator update: sector dimension above 64"; return -7; }
    long long total_groups = 0;
    std::vector<std::vector<int>> groups;   // per tile-group: job indices (same oc)
    for (size_t i = 0; i < order.size();) {
      std::vector<int> g;
      const int oc = js[order[i]].oc;
      while (i < order.size() && js[order[i]].oc == oc && (int)g.size() < 128 / slot) g.push_back(order[i++]);
      groups.push_back(g);
      total_groups += 1;
    }
    long long row_work = 0;
    for (const auto& g : groups) row_work += L.sec_rows[js[g[0]].oc];
    // about 8 CTAs' worth of K ranges per SM over the whole launch
    const long long target = 8LL * 152;
    long long kr = std::max<long long>(256, (row_work + target - 1) / target);
    kr = (kr + 31) / 32 * 32;
    long long part_off = 0;
    std::vector<int> job_parts(js.size(), 1);
    std::vector<long long> job_off(js.size(), 0);
    for (const auto& g : groups) {
      const int oc = js[g[0]].oc;
      const int rows = L.sec_rows[oc];
      const int parts = (int)((rows + kr - 1) / kr);
      const int tile0 = (int)op.tiles.size();
      for (int p = 0; p < parts; ++p) {
        OzTile t{};
        t.b_off = L.sec_off[oc];
        t.b_ld = P.dim[oc];
        t.n = P.dim[oc];
        t.r0 = (int)(p * kr);
        t.r1 = (int)std::min<long long>(rows, (p + 1) * kr);
        t.job_begin = (int)op.jobs.size();
        t.job_end = t.job_begin + (int)g.size();
        t.slot = slot;
        t.part = p;
        op.tiles.push_back(t);
      }
      (void)tile0;
      for (int j : g) {
        OzJob oj{};
        oj.map = js[j].map;
        oj.a_off = L.sec_off[js[j].ic];
        oj.a_ld = P.dim[js[j].ic];
        oj.cols = P.dim[js[j].ic];
        oj.part_off = part_off;
        job_off[j] = part_off;
        job_parts[j] = parts;
        part_off += (long long)parts * oj.cols * P.dim[oc];
        op.jobs.push_back(oj);
        op.flops += 2.0 * (double)js[j].nnz * P.dim[oc] * P.dim[js[j].ic];
      }
    }
    op.partial_elems = part_off;
    // outputs: one per operator block, its jobs in job order
    std::map<std::pair<double*, long long>, std::vector<int>> by_block;
    for (size_t j = 0; j < js.size(); ++j) {
      const long long boff = (long long)P.offset(js[j].oc) * dim + P.offset(js[j].ic);
      by_block[{js[j].O, boff}].push_back((int)j);
    }
    for (auto& kv : by_block) {
      const J& j0 = js[kv.second[0]];
      OzOut o{};
      o.O = kv.first.first + kv.first.second;
      o.ld = dim;
      o.rows = P.dim[j0.oc];
      o.cols = P.dim[j0.ic];
      o.sum_begin = (int)op.sums.size();
      for (int j : kv.second) {
        OzSum sm{};
        sm.off = job_off[j];
        sm.part_stride = (long long)P.dim[js[j].ic] * P.dim[js[j].oc];
        sm.n_parts = job_parts[j];
        sm.alpha = js[j].alpha;
        op.sums.push_back(sm);
      }
      o.sum_end = (int)op.sums.size();
      op.outs.push_back(o);
    }
    grow_upload(op.d_tiles, op.cap[0], op.tiles, stream_);
    grow_upload(op.d_jobs, op.cap[1], op.jobs, stream_);
    grow_upload(op.d_outs, op.cap[2], op.outs, stream_);
    grow_upload(op.d_sums, op.cap[3], op.sums, stream_);
    if (op.partial_elems > oz_partial_elems_) {
      cudaStreamSynchronize(stream_);
      if (oz_partial_) { untrack(oz_partial_); cudaFree(oz_partial_); }
      oz_partial_elems_ = op.partial_elems + op.partial_elems / 4;
      device_alloc((void**)&oz_partial_, oz_partial_elems_ * sizeof(double), "digit-plane partial sums");
      track(oz_partial_, oz_partial_elems_ * sizeof(double));
    }
    it = oz_cache_.emplace(node, std::move(pl)).first;
  }
  OzPlan& op = *it->second;
  launch_oz_slice(T_[node], L.size, d_scal_ + kOzAmax, oz_planes_, stream_);
  const int rc = launch_oz_gram(op.d_tiles, (int)op.tiles.size(), op.d_jobs, oz_planes_, op.npad, oz_partial_,
                                op.d_outs, (int)op.outs.size(), op.d_sums, d_err_, stream_, wait_polls);
  if (rc) { err_ = "digit-plane operator update: unsupported shape"; return rc; }
  ops_flops_ += op.flops;
  return check(cudaGetLastError(), "digit-plane operator update") ? 0 : -3;
}

// Environment operators of the bond above `node`, from its parent's tensor
// (isometric towards `node`), the sibling's up operators and the parent's
// environment operators.
int Engine::compute_down(int node) {
  const TreeNode& nd = nodes_[node];
  const int par = nd.parent;
  const TreeNode& pn = nodes_[par];
  const int leg = (pn.child_kind[0] == 1 && pn.child[0] == node) ? 0 : 1;
  const int sib_leg = 1 - leg;
  const int sib = leg_node(par, sib_leg);
  const Layout& L = layout_[par];
  const int dim = L.leg[leg].total();
  const long long dd = (long long)dim * dim;
  BondOps& out = down_[node];
  for (int c = 0; c < N_CLASSES; ++c)
    if (!out.H[c]) out.H[c] = (double*)dalloc(dd * sizeof(double));
  if (!out.Htot) out.Htot = (double*)dalloc(dd * sizeof(double));
  std::vector<char> comp_par(lat_.n_sites(), 1);
  for (int s : pn.sites) comp_par[s] = 0;
  const bool par_root = pn.parent < 0;
  struct Job { double* O; double alpha; const double* S; int shS; const double* P; int shP; };
  std::vector<Job> jobs;
  auto op_ptr = [&](int key, int shift) -> double* {
    auto it = out.term.find(key);
    if (it == out.term.end()) {
      BondOp b;
      b.ptr = (double*)dalloc(dd * sizeof(double));
      it = out.term.emplace(key, b).first;
    }
    it->second.shift = shift;
    return it->second.ptr;
  };
  for (int k = 0; k < (int)terms_.size(); ++k) {
    const bool ts = sib >= 0 ? touches(k, sib) : false;
    const bool tp = touches_sites(k, comp_par);
    if (crosses(k, node)) {
      Job j{nullptr, 1.0, nullptr, 0, nullptr, 0};
      if (ts) { const BondOp& b = up_[sib].term.at(k); j.S = b.ptr; j.shS = b.shift; }
      if (tp) { const BondOp& b = down_[par].term.at(k); j.P = b.ptr; j.shP = b.shift; }
      const int dz = j.shS - j.shP;
      j.O = op_ptr(k, -dz);
      jobs.push_back(j);
    } else if (!touches(k, node) && ts && tp) {
      // inside the complement, crossing sibling | outside-parent
      const BondOp& b1 = up_[sib].term.at(k);
      const BondOp& b2 = down_[par].term.at(k);
      jobs.push_back({out.H[terms_[k].cls], terms_[k].coef, b1.ptr, b1.shift, b2.ptr, b2.shift});
    }
  }
  for (int cl = 0; cl < N_CLASSES; ++cl) {
    jobs.push_back({out.H[cl], 1.0, up_[sib].H[cl], 0, nullptr, 0});
    if (!par_root) jobs.push_back({out.H[cl], 1.0, nullptr, 0, down_[par].H[cl], 0});
  }
  for (int c = 0; c < N_CLASSES; ++c) cudaMemsetAsync(out.H[c], 0, dd * sizeof(double), stream_);
  for (auto& kv : out.term) cudaMemsetAsync(kv.second.ptr, 0, dd * sizeof(double), stream_);
  long long zsize = 0;
  std::map<int, Layout> lays;
  for (int s = -2; s <= 2; ++s) {
    lays[s] = shifted(par, s);
    zsize = std::max(zsize, lays[s].size);
  }
  const int batch = std::max<int>(1, (int)std::min<long long>((long long)jobs.size(), kZPoolBudget / (2 * std::max(1LL, zsize))));
  ensure_zpool(2 * batch * zsize);
  const int ds = L.leg[sib_leg].total(), dp = L.leg[2].total();
  const double* T = T_[par];
  int rc = 0;
  for (size_t j0 = 0, bi = 0; j0 < jobs.size() && rc == 0; j0 += batch, ++bi) {
    const size_t j1 = std::min(jobs.size(), j0 + batch);
    cudaMemsetAsync(zpool_, 0, 2 * batch * zsize * sizeof(double), stream_);
    KPlan* st[3];
    cached_plans(PK_DOWN, node, (int)bi, 3, st, [&](KPlan** p) {
      for (size_t j = j0; j < j1; ++j) {
        const Job& jb = jobs[j];
        double* z1 = zpool_ + (2 * (j - j0)) * zsize;
        double* z2 = z1 + zsize;
        const double* Z;
        int shift;
        // sibling op on sib_leg: layout shift += shS; parent-leg op: shift -= shP
        if (jb.S && jb.P) {
          plan_leg_apply(*p[0], L, T, lays[jb.shS], z1, sib_leg, jb.S, ds, jb.shS, false, 1.0);
          plan_leg_apply(*p[1], lays[jb.shS], z1, lays[jb.shS - jb.shP], z2, 2, jb.P, dp, jb.shP, false, 1.0);
          Z = z2;
          shift = jb.shS - jb.shP;
        } else if (jb.S) {
          plan_leg_apply(*p[0], L, T, lays[jb.shS], z1, sib_leg, jb.S, ds, jb.shS, false, 1.0);
          Z = z1;
          shift = jb.shS;
        } else {
          plan_leg_apply(*p[0], L, T, lays[-jb.shP], z1, 2, jb.P, dp, jb.shP, false, 1.0);
          Z = z1;
          shift = -jb.shP;
        }
        plan_contract_but(*p[2], L, T, lays[shift], Z, leg, jb.O, dim, jb.alpha);
      }
    });
    for (int i = 0; i < 3 && rc == 0; ++i) rc = launch_plan(st[i], ops_mode());
  }
  cudaMemsetAsync(out.Htot, 0, dd * sizeof(double), stream_);
  for (int c = 0; c < N_CLASSES; ++c) launch_add_scaled(out.H[c], out.Htot, dd, 1.0, stream_);
  return rc;
}

// ------------------------------------------------------------------ centre moves
int Engine::move_to(int target) {
  if (target == center_) return 0;
  cudaEvent_t e0 = nullptr;
  if (profiling_) ev_begin(&e0);
  int rc = move_path(target);
  if (profiling_) ev_end(e0, KC_MOVE, 0, 0, 0);
  return rc;
}

int Engine::move_path(int target) {
  // path from centre to target through the lowest common ancestor
  std::vector<int> pa, pb;
  for (int x = center_; x >= 0; x = nodes_[x].parent) pa.push_back(x);
  for (int x = target; x >= 0; x = nodes_[x].parent) pb.push_back(x);
  int common = -1;
  for (int x : pa)
    if (std::find(pb.begin(), pb.end(), x) != pb.end()) { common = x; break; }
  std::vector<int> path;
  for (int x : pa) { path.push_back(x); if (x == common) break; }
  std::vector<int> down;
  for (int x : pb) { if (x == common) break; down.push_back(x); }
  for (auto it = down.rbegin(); it != down.rend(); ++it) path.push_back(*it);
  for (size_t i = 1; i < path.size(); ++i) {
    const int c = path[i - 1], t = path[i];
    int leg_c, leg_t;
    if (nodes_[c].parent == t) {
      leg_c = 2;
      leg_t = (nodes_[t].child_kind[0] == 1 && nodes_[t].child[0] == c) ? 0 : 1;
    } else {
      leg_t = 2;
      leg_c = (nodes_[c].child_kind[0] == 1 && nodes_[c].child[0] == t) ? 0 : 1;
    }
    cudaEvent_t e0 = nullptr;
    if (profiling_) ev_begin(&e0);
    int rc = qr_toward(c, leg_c, move_R_);
    if (!rc) rc = absorb(t, leg_t, move_R_);
    if (rc) return rc;
    if (profiling_) ev_end(e0, KC_MOVE_QR, 0, 0, 0);
    center_ = t;
    tc_w_node_ = -1;   // environment operators change with the move
    if (profiling_) ev_begin(&e0);
    ops_flops_ = 0.0;
    const bool bottom_up = leg_c == 2 && nodes_[c].child_kind[0] == 0;
    if (leg_c == 2) rc = compute_up(c);
    else rc = compute_down(t);
    if (rc) return rc;
    if (profiling_) ev_end(e0, bottom_up ? KC_MOVE_OPS_BOTTOM : KC_MOVE_OPS, ops_flops_, ops_flops_, 0);
  }
  return check(cudaGetLastError(), "move") ? 0 : -3;
}

// ------------------------------------------------------------------ H_eff
// Terms of H_eff at `node` (Methods step (i)): block Hamiltonians of the
// three legs and every term touching at least two of the three regions.
void Engine::build_heff_terms(int node, int cls, std::vector<HTerm>* out) {
  out->clear();
  const TreeNode& nd = nodes_[node];
  const bool bottom = nd.child_kind[0] == 0;
  std::vector<char> comp(lat_.n_sites(), 1);
  for (int s : nd.sites) comp[s] = 0;
  const bool root = nd.parent < 0;
  for (int leg = 0; leg < 2; ++leg) {
    HTerm h;
    h.cls = cls;
    if (bottom) {
      h.op[leg].kind = 2;
      h.op[leg].term = -1;
      h.op[leg].cls = cls;
    } else {
      const BondOps& b = up_[leg_node(node, leg)];
      h.op[leg].kind = 1;
      h.op[leg].ptr = cls < 0 ? b.Htot : b.H[cls];
    }
    out->push_back(h);
  }
  if (!root) {
    HTerm h;
    h.cls = cls;
    h.op[2].kind = 1;
    h.op[2].ptr = cls < 0 ? down_[node].Htot : down_[node].H[cls];
    out->push_back(h);
  }
  for (int k = 0; k < (int)terms_.size(); ++k) {
    if (cls >= 0 && terms_[k].cls != cls) continue;
    bool t[3] = {false, false, false};
    for (auto& so : terms_[k].ops) {
      for (int leg = 0; leg < 2; ++leg) {
        int cn = leg_node(node, leg);
        bool in = cn >= 0 ? in_region_[cn][so.first] : so.first == leg_site(node, leg);
        if (in) t[leg] = true;
      }
      if (comp[so.first]) t[2] = true;
    }
    if ((int)t[0] + (int)t[1] + (int)t[2] < 2) continue;
    HTerm h;
    h.coef = terms_[k].coef;
    h.cls = terms_[k].cls;
    for (int leg = 0; leg < 2; ++leg) {
      if (!t[leg]) continue;
      if (bottom) {
        h.op[leg].kind = 2;
        h.op[leg].term = k;
      } else {
        const BondOp& b = up_[leg_node(node, leg)].term.at(k);
        h.op[leg].kind = 1;
        h.op[leg].ptr = b.ptr;
        h.op[leg].shift = b.shift;
      }
    }
    if (t[2]) {
      const BondOp& b = down_[node].term.at(k);
      h.op[2].kind = 1;
      h.op[2].ptr = b.ptr;
      h.op[2].shift = b.shift;
    }
    out->push_back(h);
  }
}

// H_eff plans of (node, class filter), built on first use and replayed.
// Returns nullptr (err_ set) if validation fails.
// adjoint: the transposed operator (every term applied as A^T (x) B^T (x) C^T),
// FP64 only; cached under a separate key.
Engine::HeffPlans* Engine::heff_plans(int node, int cls, bool adjoint) {
  const auto key = std::make_pair(node, adjoint ? cls - 1000 : cls);
  auto hit = heff_cache_.find(key);
  if (hit != heff_cache_.end()) return hit->second.get();
  std::unique_ptr<HeffPlans> hp(new HeffPlans);
  KPlan* st = hp->st;
  std::vector<HTerm> hts;
  build_heff_terms(node, cls, &hts);
  const Layout& L = layout_[node];
  const bool bottom = nodes_[node].child_kind[0] == 0;
  KPlan& s3 = st[2];
  const int d2 = L.leg[2].total();
  const double cst = (cls < 0 || cls == CLS_NU) ? constant_ : 0.0;
  if (bottom && adjoint) {
    // transposed terms: the forward chunk y_oc += x_ic[map] C[oc, ic]^T becomes
    // y_ic += x_oc[inverse map] C[oc, ic]
    for (size_t oc = 0; oc < L.leg[2].q.size(); ++oc) {
      const int rows = L.sec_rows[oc];
      if (rows == 0) continue;
      const int dc = L.leg[2].dim[oc];
      s3.add_output(y_out_ + L.sec_off[oc], dc, 1, rows, dc, 0);
      if (cst != 0.0) {
        KChunk c = make_chunk();
        c.A = x_in_ + L.sec_off[oc]; c.a_m = dc; c.a_k = 1;
        c.add = 1; c.alpha = cst;
        s3.add_chunk(c);
      }
    }
    for (size_t oc = 0; oc < L.leg[2].q.size(); ++oc) {
      if (L.sec_rows[oc] == 0) continue;
      const int dco = L.leg[2].dim[oc];
      for (const HTerm& h : hts) {
        const bool phys = h.op[0].kind == 2 || h.op[1].kind == 2;
        const RowMap* rm = nullptr;
        if (phys) {
          if (h.op[0].kind == 2 && h.op[0].term < 0) rm = &site_ham_map(node, 0, h.op[0].cls)[oc];
          else if (h.op[1].kind == 2 && h.op[1].term < 0) rm = &site_ham_map(node, 1, h.op[1].cls)[oc];
          else rm = &rowmap(node, h.op[0].kind == 2 ? h.op[0].term : h.op[1].term)[oc];
          if (rm->src_sector < 0) continue;
        }
        const int ic = phys ? rm->src_sector : (int)oc;
        if (L.sec_rows[ic] == 0) continue;
        const int dci = L.leg[2].dim[ic];
        KChunk c = make_chunk();
        c.A = x_in_ + L.sec_off[oc]; c.a_m = dco; c.a_k = 1;
        if (rm) {
          const RowMap& inv = inverse_rowmap(*rm, L.sec_rows[oc], L.sec_rows[ic]);
          c.amap = inv.map; c.aval = inv.val;
        }
        c.alpha = h.coef;
        if (h.op[2].kind == 1) {
          if (L.leg[2].find(L.leg[2].q[ic] + h.op[2].shift) != (int)oc) continue;
          c.B = h.op[2].ptr + L.leg[2].offset((int)oc) * d2 + L.leg[2].offset(ic);
          c.b_k = d2; c.b_n = 1;
          c.K = dco;
        } else {
          if (ic != (int)oc) continue;
          c.add = 1;
        }
        s3.add_output(y_out_ + L.sec_off[ic], dci, 1, L.sec_rows[ic], dci, 0);
        s3.add_chunk(c);
      }
    }
  } else if (bottom) {
    // per output c-sector: chunks over terms, A rows gathered from x_in
    for (size_t oc = 0; oc < L.leg[2].q.size(); ++oc) {
      const int rows = L.sec_rows[oc];
      if (rows == 0) continue;
      const int dc = L.leg[2].dim[oc];
      s3.add_output(y_out_ + L.sec_off[oc], dc, 1, rows, dc, 0);
      if (cst != 0.0) {
        KChunk c = make_chunk();
        c.A = x_in_ + L.sec_off[oc]; c.a_m = dc; c.a_k = 1;
        c.add = 1; c.alpha = cst;
        s3.add_chunk(c);
      }
      for (const HTerm& h : hts) {
        const bool phys = h.op[0].kind == 2 || h.op[1].kind == 2;
        const RowMap* rm = nullptr;
        if (phys) {
          if (h.op[0].kind == 2 && h.op[0].term < 0) rm = &site_ham_map(node, 0, h.op[0].cls)[oc];
          else if (h.op[1].kind == 2 && h.op[1].term < 0) rm = &site_ham_map(node, 1, h.op[1].cls)[oc];
          else rm = &rowmap(node, h.op[0].kind == 2 ? h.op[0].term : h.op[1].term)[oc];
          if (rm->src_sector < 0) continue;
        }
        const int ic = phys ? rm->src_sector : (int)oc;
        const int dci = L.leg[2].dim[ic];
        KChunk c = make_chunk();
        c.A = x_in_ + L.sec_off[ic]; c.a_m = dci; c.a_k = 1;
        if (rm) { c.amap = rm->map; c.aval = rm->val; }
        c.alpha = h.coef;
        if (h.op[2].kind == 1) {
          // sanity: env op must map sector ic -> oc
          if (L.leg[2].find(L.leg[2].q[ic] + h.op[2].shift) != (int)oc) continue;
          c.B = h.op[2].ptr + L.leg[2].offset((int)oc) * d2 + L.leg[2].offset(ic);
          c.b_k = 1; c.b_n = d2;
          c.K = dci;
        } else {
          if (ic != (int)oc) continue;
          c.add = 1;
        }
        s3.add_chunk(c);
      }
    }
  } else {
    // upper node: Z buffers per term, stage 1 (first child op), stage 2 (second)
    std::map<int, Layout> lays;
    long long zsize = 0;
    for (int s = -2; s <= 2; ++s) {
      lays[s] = shifted(node, s);
      zsize = std::max(zsize, lays[s].size);
    }
    int nz = 0;
    for (const HTerm& h : hts) nz += (h.op[0].kind ? 1 : 0) + (h.op[1].kind ? 1 : 0);
    ensure_zpool(std::max(1, nz) * zsize);
    hp->z_elems = (long long)nz * zsize;
    const int dl = L.leg[0].total(), dr = L.leg[1].total();
    struct Src { const double* Z; int shift; };
    std::vector<Src> srcs;
    int zi = 0;
    // the adjoint applies each operator transposed, which reverses its shift
    const int sg = adjoint ? -1 : 1;
    for (const HTerm& h : hts) {
      const double* Z = x_in_;
      int shift = 0;
      const int sh0 = sg * h.op[0].shift, sh1 = sg * h.op[1].shift;
      if (h.op[0].kind) {
        double* z1 = zpool_ + (zi++) * zsize;
        plan_leg_apply(st[0], L, x_in_, lays[sh0], z1, 0, h.op[0].ptr, dl, sh0, adjoint, 1.0);
        Z = z1;
        shift = sh0;
        if (h.op[1].kind) {
          double* z2 = zpool_ + (zi++) * zsize;
          plan_leg_apply(st[1], lays[shift], z1, lays[shift + sh1], z2, 1, h.op[1].ptr, dr, sh1, adjoint, 1.0);
          Z = z2;
          shift += sh1;
        }
      } else if (h.op[1].kind) {
        double* z1 = zpool_ + (zi++) * zsize;
        plan_leg_apply(st[0], L, x_in_, lays[sh1], z1, 1, h.op[1].ptr, dr, sh1, adjoint, 1.0);
        Z = z1;
        shift = sh1;
      }
      srcs.push_back({Z, shift});
    }
    // stage 3: per y block, chunks over terms
    for (const Layout::Blk& yb : L.blk) {
      s3.add_output(y_out_ + yb.off, yb.dc, 1, yb.da * yb.db, yb.dc, 0);
      if (cst != 0.0) {
        KChunk c = make_chunk();
        c.A = x_in_ + yb.off; c.a_m = yb.dc; c.a_k = 1;
        c.add = 1; c.alpha = cst;
        s3.add_chunk(c);
      }
      for (size_t t = 0; t < hts.size(); ++t) {
        const HTerm& h = hts[t];
        const Layout& LZ = lays[srcs[t].shift];
        const int k = LZ.find(yb.ia, yb.ib);
        if (k < 0) continue;
        const Layout::Blk& zb = LZ.blk[k];
        KChunk c = make_chunk();
        c.A = srcs[t].Z + zb.off; c.a_m = zb.dc; c.a_k = 1;
        c.alpha = h.coef;
        if (h.op[2].kind == 1 && adjoint) {
          // C^T: y_c' = sum_c C[c, c'] Z_c, C mapping sector yb.ic to zb.ic
          if (L.leg[2].find(L.leg[2].q[yb.ic] + h.op[2].shift) != zb.ic) continue;
          c.B = h.op[2].ptr + L.leg[2].offset(zb.ic) * d2 + L.leg[2].offset(yb.ic);
          c.b_k = d2; c.b_n = 1;
          c.K = zb.dc;
        } else if (h.op[2].kind == 1) {
          if (L.leg[2].find(L.leg[2].q[zb.ic] + h.op[2].shift) != yb.ic) continue;
          c.B = h.op[2].ptr + L.leg[2].offset(yb.ic) * d2 + L.leg[2].offset(zb.ic);
          c.b_k = 1; c.b_n = d2;
          c.K = zb.dc;
        } else {
          if (zb.ic != yb.ic) continue;
          c.add = 1;
        }
        s3.add_chunk(c);
      }
    }
    for (int i = 0; i < 2; ++i) st[i].finalize(kKPart);
  }
  s3.finalize(kKPart);
  for (int i = 0; i < 3; ++i) hp->flops += st[i].flops;
  if (!check(cudaGetLastError(), "plan")) return nullptr;
  HeffPlans* raw = hp.get();
  heff_cache_[key] = std::move(hp);
  return raw;
}

bool Engine::mixed_node(int node) const {
  (void)node;
  return precision_ != PREC_FP64;
}

int Engine::apply_heff(const double* x, double* y, int cls) {
  const long long n = layout_[center_].size;
  const bool bottom = nodes_[center_].child_kind[0] == 0;
  if (use_mixed_ && cls < 0 && bottom) {
    if (x != x_in_) launch_copy(x, x_in_, n, stream_);
    int rc = apply_heff_mixed();
    if (rc) return rc;
    if (y != y_out_) launch_copy(y_out_, y, n, stream_);
    return check(cudaGetLastError(), "apply_heff (mixed)") ? 0 : -3;
  }
  if (use_mixed_ && cls < 0) {
    // upper node in a mixed state: tensor-core leg contractions
    if (x != x_in_) launch_copy(x, x_in_, n, stream_);
    int rc = apply_heff_tg();
    if (rc) return rc;
    if (y != y_out_) launch_copy(y_out_, y, n, stream_);
    return 0;
  }
  HeffPlans* hp = heff_plans(center_, cls, false);
  if (!hp) return -1;
  if (x != x_in_) launch_copy(x, x_in_, n, stream_);
  cudaEvent_t e0 = nullptr;
  if (profiling_) ev_begin(&e0);
  if (!bottom && hp->z_elems > 0) {
    // Z blocks that no source block maps to must read as zero
    cudaMemsetAsync(zpool_, 0, hp->z_elems * sizeof(double), stream_);
  }
  for (int i = 0; i < 3; ++i) {
    const int rc = launch_kplan(hp->st[i], ff_products_ && cls < 0 ? 2 : 0, true);
    if (rc) return rc;
  }
  if (profiling_) ev_end(e0, bottom ? KC_HEFF_SIMT_BOTTOM : KC_HEFF_SIMT_UPPER, hp->flops, hp->flops, 0.0);
  if (y != y_out_) launch_copy(y_out_, y, n, stream_);
  return check(cudaGetLastError(), "apply_heff") ? 0 : -3;
}

// y = H_eff^T x at the current centre: the hand-written adjoint of the
// contraction (each term transposed), FP64.  H_eff is symmetric, so this
// equals apply_heff up to rounding; the energy gradient uses both.
int Engine::apply_heff_adjoint(const double* x, double* y) {
  const long long n = layout_[center_].size;
  const bool bottom = nodes_[center_].child_kind[0] == 0;
  HeffPlans* hp = heff_plans(center_, -1, true);
  if (!hp) return -1;
  if (x != x_in_) launch_copy(x, x_in_, n, stream_);
  if (!bottom && hp->z_elems > 0) cudaMemsetAsync(zpool_, 0, hp->z_elems * sizeof(double), stream_);
  for (int i = 0; i < 3; ++i) {
    const int rc = launch_kplan(hp->st[i], 0, true);
    if (rc) return rc;
  }
  if (y != y_out_) launch_copy(y_out_, y, n, stream_);
  return check(cudaGetLastError(), "apply_heff_adjoint") ? 0 : -3;
}

// E(psi) = psi^T H_eff psi / psi^T psi at the centre (psi = the centre tensor
// when psi == nullptr).  grad (device, optional) = dE/dpsi = ((H + H^T) psi -
// 2 E psi) / psi^T psi.  dE/dc per coupling class: E is linear in the
// couplings (Eq. (1) + Eq. (16)), so dE/dc = <psi|H_c|psi> / (c <psi|psi>),
// the Hellmann-Feynman value; NaN where the coupling is zero (its terms are
// not in the model).  Every product runs in FP64.
int Engine::energy_grad(const double* psi, double* energy, double* grad, double dc[N_CLASSES]) {
  const long long n = layout_[center_].size;
  const double* x = psi ? psi : T_[center_];
  double* hx = grad_a_;
  double* htx = grad_b_;
  double* dv = d_scal_ + 700;   // [0] |psi|^2, [1] psi.H psi, [2..7] classes
  int rc = 0;
  launch_dot(x, x, n, d_partial_, dv, stream_);
  if ((rc = apply_heff(x, hx, -1))) return rc;
  launch_dot(x, hx, n, d_partial_, dv + 1, stream_);
  for (int c = 0; c < N_CLASSES; ++c) {
    if ((rc = apply_heff(x, y_out_, c))) return rc;
    launch_dot(x, y_out_, n, d_partial_, dv + 2 + c, stream_);
  }
  double host[2 + N_CLASSES];
  cudaMemcpyAsync(host, dv, (2 + N_CLASSES) * sizeof(double), cudaMemcpyDeviceToHost, stream_);
  if (!check(cudaStreamSynchronize(stream_), "energy gradient")) return -3;
  const double nrm = host[0];
  if (!(nrm > 0.0)) { err_ = "energy gradient: zero vector"; return -1; }
  const double e = host[1] / nrm;
  if (energy) *energy = e;
  // the chemical potentials have no single coupling: dc[CLS_MU] = <H_mu>
  const double coupling[N_CLASSES] = {p_.t, p_.m, p_.ge2, p_.cB, p_.nu, 1.0};
  for (int c = 0; c < N_CLASSES; ++c)
    dc[c] = coupling[c] != 0.0 ? host[2 + c] / nrm / coupling[c] : std::nan("");
  if (grad) {
    if ((rc = apply_heff_adjoint(x, htx))) return rc;
    // grad = (hx + htx - 2 e x) / nrm
    launch_add_scaled(htx, hx, n, 1.0, stream_);
    launch_copy(hx, grad, n, stream_);
    launch_axpby(x, grad, n, nullptr, -2.0 * e / nrm, 1.0, nullptr, 1.0 / nrm, stream_);
    if (!check(cudaStreamSynchronize(stream_), "energy gradient")) return -3;
  }
  return check(cudaGetLastError(), "energy gradient") ? 0 : -3;
}

// One gradient step on the centre tensor: psi <- (psi - eta dE/dpsi) /
// |psi - eta dE/dpsi|, energies before and after.
int Engine::gradient_step(double eta, double* e_before, double* e_after) {
  const long long n = layout_[center_].size;
  double dc[N_CLASSES];
  double e0 = 0.0;
  int rc = energy_grad(nullptr, &e0, grad_c_, dc);
  if (rc) return rc;
  launch_axpby(grad_c_, T_[center_], n, nullptr, -eta, 1.0, nullptr, 1.0, stream_);
  double* nrm2 = d_scal_ + 640;
  launch_dot(T_[center_], T_[center_], n, d_partial_, nrm2, stream_);
  launch_scale_inv_sqrt(T_[center_], T_[center_], n, nrm2, stream_);
  double e1 = 0.0;
  rc = energy_grad(nullptr, &e1, nullptr, dc);
  if (rc) return rc;
  if (e_before) *e_before = e0;
  if (e_after) *e_after = e1;
  return 0;
}

// ------------------------------------------------------------------ mixed precision
// Tensor-core plan of a bottom node: environment-coupled terms (and the
// environment block Hamiltonian) become GEMM chunks with their operator
// blocks converted to BF16 / FP32 and scaled by the term coefficient; terms
// acting on the two sites only, and the constant, are FP64 epilogue adds.
TcPlan* Engine::tc_plan(int node) {
  auto cit = tc_cache_.find(node);
  if (cit != tc_cache_.end()) return cit->second.get();
  std::vector<HTerm> hts;
  build_heff_terms(node, -1, &hts);
  const Layout& L = layout_[node];
  const Sectors& P = L.leg[2];
  const int ns = (int)P.q.size();
  const int d2 = P.total();
  const int elem = precision_ == PREC_BF16 ? 2 : 4;
  const bool split = precision_ == PREC_TF32X3;
  const int xmul = split ? 2 : 1;   // staged row width in units of kpad
  const int kmul = split ? 2 : 1;   // staged B row width in units of kpad
  std::unique_ptr<TcPlan> tp(new TcPlan);
  TcPlan& tc = *tp;
  std::vector<long long> soff(ns, 0);
  std::vector<int> kpad(ns);
  long long xs = 0;
  for (int i = 0; i < ns; ++i) {
    kpad[i] = (P.dim[i] + 15) / 16 * 16;
    soff[i] = xs;
    xs += (long long)L.sec_rows[i] * kpad[i];
  }
  // operand staging holds xmul * xs elements; an FP32 copy (xs) serves the epilogue
  if (xs > xstage_elems_) {
    clear_tc_cache();   // cached plans point into the old staging
    if (xstage_) { untrack(xstage_); cudaFree(xstage_); }
    if (xstage32_) { untrack(xstage32_); cudaFree(xstage32_); xstage32_ = nullptr; }
    xstage_elems_ = xs + xs / 4;
    if (!check(cudaMalloc(&xstage_, 2 * xstage_elems_ * elem), "x staging")) return nullptr;
    track(xstage_, 2 * xstage_elems_ * elem);
    if (!check(cudaMalloc(&xstage32_, xstage_elems_ * 4), "x staging")) return nullptr;
    track(xstage32_, xstage_elems_ * 4);
  }
  float* x32 = xstage32_;
  for (int i = 0; i < ns; ++i) {
    if (L.sec_rows[i] == 0) continue;
    ConvJob j;
    j.src = x_in_ + L.sec_off[i];
    j.ld_src = P.dim[i];
    j.cs_src = 1;
    j.dst = (char*)xstage_ + xmul * soff[i] * elem;
    j.dst32 = xstage32_ + soff[i];
    j.rows = L.sec_rows[i];
    j.cols = P.dim[i];
    j.kpad = kpad[i];
    j.scale = 1.0;
    tc.xjobs.push_back(j);
    tc.x_max_elems = std::max(tc.x_max_elems, (long long)j.rows * j.kpad);
  }
  // W slots
  long long wtot = 0;
  struct WJ { int oc, ic; const double* op; double coef; long long off; };
  std::vector<WJ> wj;
  const double cst = constant_;
  for (int oc = 0; oc < ns; ++oc) {
    const int rows = L.sec_rows[oc];
    if (rows == 0) continue;
    TcOutput o;
    o.y = y_out_ + L.sec_off[oc];
    o.rows = rows;
    o.n = P.dim[oc];
    o.npad = kpad[oc];
    o.chunk_begin = (int)tc.chunks.size();
    o.add_begin = (int)tc.adds.size();
    tc.max_npad = std::max(tc.max_npad, o.npad);
    if (cst != 0.0) {
      TcAdd a;
      a.X32 = x32 + soff[oc];
      a.map = nullptr;
      a.val = nullptr;
      a.alpha = cst;
      a.ld = kpad[oc];
      tc.adds.push_back(a);
    }
    for (const HTerm& h : hts) {
      const bool phys = h.op[0].kind == 2 || h.op[1].kind == 2;
      const RowMap* rm = nullptr;
      if (phys) {
        if (h.op[0].kind == 2 && h.op[0].term < 0) rm = &site_ham_map(node, 0, h.op[0].cls)[oc];
        else if (h.op[1].kind == 2 && h.op[1].term < 0) rm = &site_ham_map(node, 1, h.op[1].cls)[oc];
        else rm = &rowmap(node, h.op[0].kind == 2 ? h.op[0].term : h.op[1].term)[oc];
        if (rm->src_sector < 0) continue;
      }
      const int ic = phys ? rm->src_sector : oc;
      if (h.op[2].kind == 1) {
        if (P.find(P.q[ic] + h.op[2].shift) != oc) continue;
        if (rm && rm->val) {   // GEMM terms carry +-1 maps only
          err_ = "tensor-core plan: valued row map on an environment term";
          return nullptr;
        }
        TcChunk c;
        c.X = (char*)xstage_ + xmul * soff[ic] * elem;
        c.map = rm ? rm->map : nullptr;
        c.kpad = kmul * kpad[ic];
        c.xstride = xmul * kpad[ic];
        const long long welems = (long long)o.npad * c.kpad;
        wj.push_back({oc, ic, h.op[2].ptr, h.coef, wtot});
        c.W = (const void*)(intptr_t)wtot;   // patched below once the buffer exists
        wtot += welems;
        tc.chunks.push_back(c);
        tc.max_kpad = std::max(tc.max_kpad, c.kpad);
        const double nnz = rm ? (double)rm->nnz : (double)rows;
        tc.flops_alg += 2.0 * nnz * P.dim[oc] * P.dim[ic];
        tc.flops_exec += 2.0 * ((rows + 127) / 128 * 128) * o.npad * kpad[ic] * (split ? 3 : 1);
      } else {
        if (ic != oc) continue;
        TcAdd a;
        a.X32 = x32 + soff[ic];
        a.map = rm ? rm->map : nullptr;
        a.val = rm ? rm->val : nullptr;
        a.alpha = h.coef;
        a.ld = kpad[ic];
        tc.adds.push_back(a);
      }
    }
    o.chunk_end = (int)tc.chunks.size();
    o.add_end = (int)tc.adds.size();
    tc.outs.push_back(o);
    for (int r0 = 0; r0 < rows; r0 += 128) tc.tiles.push_back({(int)tc.outs.size() - 1, r0});
  }
  if (wtot > wbuf_elems_) {
    clear_tc_cache();   // cached plans point into the old W buffer
    if (wbuf_) { untrack(wbuf_); cudaFree(wbuf_); }
    wbuf_elems_ = wtot + wtot / 4 + 1024;
    if (!check(cudaMalloc(&wbuf_, wbuf_elems_ * elem), "W staging")) return nullptr;
    track(wbuf_, wbuf_elems_ * elem);
  }
  for (TcChunk& c : tc.chunks) c.W = (char*)wbuf_ + (intptr_t)c.W * elem;
  tc.wtot = wtot;
  for (const WJ& w : wj) {
    ConvJob j;
    j.src = w.op + P.offset(w.oc) * (long long)d2 + P.offset(w.ic);
    j.ld_src = d2;
    j.cs_src = 1;
    j.dst = (char*)wbuf_ + w.off * elem;
    j.dst32 = nullptr;
    j.rows = P.dim[w.oc];
    j.cols = P.dim[w.ic];
    j.kpad = kpad[w.ic];
    j.scale = w.coef;
    tc.wjobs.push_back(j);
    tc.w_max_elems = std::max(tc.w_max_elems, (long long)j.rows * j.kpad);
  }
  // algorithmic bytes: x staging read once, y written once (FP64), W read once
  tc.bytes_alg = (double)xs * xmul * elem + (double)L.size * 8.0 + (double)wtot * elem;
  grow_upload(tc.d_tiles, tc.cap[0], tc.tiles, stream_);
  grow_upload(tc.d_outs, tc.cap[1], tc.outs, stream_);
  grow_upload(tc.d_chunks, tc.cap[2], tc.chunks, stream_);
  grow_upload(tc.d_adds, tc.cap[3], tc.adds, stream_);
  grow_upload(tc.d_xjobs, tc.cap[4], tc.xjobs, stream_);
  grow_upload(tc.d_wjobs, tc.cap[5], tc.wjobs, stream_);
  if (!check(cudaGetLastError(), "tc plan")) return nullptr;
  TcPlan* raw = tp.get();
  tc_cache_[node] = std::move(tp);
  return raw;
}

void Engine::clear_tc_cache() {
  cudaStreamSynchronize(stream_);
  ++gen_;
  tc_cache_.clear();
  tc_w_node_ = -1;
}

// Tensor-core plan of the centre with its environment blocks staged.
TcPlan* Engine::tc_prepare() {
  TcPlan* tc = tc_plan(center_);
  if (!tc) return nullptr;
  const int elem = precision_ == PREC_BF16 ? 2 : 4;
  const int split = precision_ == PREC_TF32X3 ? 1 : 0;
  if (tc_w_node_ != center_) {
    // environment blocks of this centre (padding zero) into the shared W buffer
    if (tc->wtot > 0) cudaMemsetAsync(wbuf_, 0, tc->wtot * elem, stream_);
    launch_convert(elem, split ? 2 : 0, tc->d_wjobs, (int)tc->wjobs.size(), tc->w_max_elems, stream_);
    tc_w_node_ = center_;
  }
  return tc;
}

int Engine::apply_heff_mixed() {
  TcPlan* tc = tc_prepare();
  if (!tc) return -1;
  const int elem = precision_ == PREC_BF16 ? 2 : 4;
  const int split = precision_ == PREC_TF32X3 ? 1 : 0;
  launch_convert(elem, split, tc->d_xjobs, (int)tc->xjobs.size(), tc->x_max_elems, stream_);
  cudaEvent_t e0 = nullptr;
  if (profiling_) ev_begin(&e0);
  int rc = launch_tc_heff(elem, split, tc->d_tiles, (int)tc->tiles.size(), tc->d_outs, tc->d_chunks, tc->d_adds,
                          tc->max_kpad, tc->max_npad, d_err_, stream_, wait_polls);
  if (rc) {
    err_ = "tensor-core H_eff: tile shape outside the supported range";
    return rc;
  }
  if (profiling_) ev_end(e0, KC_TC_HEFF, tc->flops_alg, tc->flops_exec, tc->bytes_alg);
  return 0;
}

// ------------------------------------------------------------------ tensor-core upper-node products
namespace {
constexpr int kTgRowsBig = 1 << 30;   // row split that keeps the row index linear

// Cut an output into 128-row tiles; a long chunk list is split into parts
// (partial sums added afterwards) when the plan has few tiles.
void tg_tiles(TgPlan& pl, int oi, int parts_wanted) {
  TgOut& o = pl.outs[oi];
  const int cb = o.n_parts, ce = (int)pl.chunks.size();   // n_parts holds chunk_begin while building
  long long steps = 0;
  for (int c = cb; c < ce; ++c) steps += (pl.chunks[c].K + 31) / 32;
  int parts = 1;
  if (parts_wanted > 1 && steps >= 8) parts = (int)std::min<long long>(parts_wanted, steps / 4);
  std::vector<std::pair<int, int>> ranges;
  if (parts <= 1) {
    ranges.push_back({cb, ce});
  } else {
    const long long per = (steps + parts - 1) / parts;
    long long acc = 0;
    int start = cb;
    for (int c = cb; c < ce; ++c) {
      acc += (pl.chunks[c].K + 31) / 32;
      if (acc >= per && c + 1 < ce) { ranges.push_back({start, c + 1}); start = c + 1; acc = 0; }
    }
    ranges.push_back({start, ce});
  }
  o.n_parts = (int)ranges.size();
  if (o.n_parts > 1) {
    o.part_off = pl.scratch_need;
    pl.scratch_need += (long long)o.n_parts * o.rows * o.N;
    pl.red.push_back(oi);
  }
  for (int r0 = 0; r0 < o.rows; r0 += 128)
    for (size_t p = 0; p < ranges.size(); ++p)
      pl.tiles.push_back(TgTile{oi, r0, ranges[p].first, ranges[p].second, o.n_parts > 1 ? (int)p : -1});
}
}  // namespace

// Plans of the mixed-precision upper-node product at `node`.  Every term's
// operators on the two child legs are applied first (stage 0: the first one,
// stage 1: the second one when a term has both), into FP32 intermediates that
// keep the (a, b, c) element order of their blocks; stage 2 then forms every
// output block of y as one K-concatenated sum over terms of the intermediate
// (or x) times the term's parent-leg operator block, or times the identity
// when the term has none there (the constant of Eq. (16) likewise).
Engine::TgHeff* Engine::tg_plans(int node) {
  auto it = tg_cache_.find(node);
  if (it != tg_cache_.end()) return it->second.get();
  std::vector<HTerm> hts;
  build_heff_terms(node, -1, &hts);
  const Layout& L = layout_[node];
  std::map<int, Layout> lays;
  long long zsize = 0;
  for (int sh = -2; sh <= 2; ++sh) {
    lays[sh] = shifted(node, sh);
    zsize = std::max(zsize, lays[sh].size);
  }
  int nz = 0;
  for (const HTerm& h : hts) nz += (h.op[0].kind ? 1 : 0) + (h.op[1].kind ? 1 : 0);
  if ((long long)nz * zsize > tg_pool_elems_) {
    cudaStreamSynchronize(stream_);   // cached plans point into the old pool
    tg_cache_.clear();
    ++gen_;
    if (tg_pool_) { untrack(tg_pool_); cudaFree(tg_pool_); tg_pool_ = nullptr; }
    tg_pool_elems_ = (long long)std::max(nz, 1) * zsize + zsize;
    device_alloc((void**)&tg_pool_, tg_pool_elems_ * sizeof(float), "tensor-core intermediates");
    track(tg_pool_, tg_pool_elems_ * sizeof(float));
  }
  const int d0 = L.leg[0].total(), d1 = L.leg[1].total(), d2 = L.leg[2].total();
  int dmax = 1;
  for (const Sectors& b : bonds_) dmax = std::max(dmax, b.total());
  dmax = std::max(dmax, std::max(d0, std::max(d1, d2)));
  if (dmax > ident_dim_) {
    cudaStreamSynchronize(stream_);   // cached plans point at the old identity
    tg_cache_.clear();
    ++gen_;
    if (ident_) { untrack(ident_); cudaFree(ident_); }
    ident_dim_ = dmax;
    device_alloc((void**)&ident_, (size_t)dmax * dmax * sizeof(double), "identity blocks");
    track(ident_, (size_t)dmax * dmax * sizeof(double));
    std::vector<double> h((size_t)dmax * dmax, 0.0);
    for (int i = 0; i < dmax; ++i) h[(size_t)i * dmax + i] = 1.0;
    cudaMemcpyAsync(ident_, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, stream_);
    cudaStreamSynchronize(stream_);
  }
  std::unique_ptr<TgHeff> tp(new TgHeff);
  TgHeff& T = *tp;
  // Z = op (x)_leg X on the child legs, block by block; written[] marks the
  // output blocks that receive a source block (the others are never read)
  auto leg_apply = [&](TgPlan& pl, const Layout& LX, const void* X, bool x_f32, const std::vector<char>* xw,
                       const Layout& LY, float* Y, std::vector<char>* yw, int leg, const OpRef& op, int shiftP,
                       int dimP) {
    const Sectors& S = LX.leg[leg];
    for (size_t bi = 0; bi < LX.blk.size(); ++bi) {
      if (xw && !(*xw)[bi]) continue;
      const Layout::Blk& b = LX.blk[bi];
      const int src = leg == 0 ? b.ia : b.ib;
      const int dst = S.find(S.q[src] + shiftP);
      if (dst < 0) continue;
      const int k = LY.find(leg == 0 ? dst : b.ia, leg == 0 ? b.ib : dst);
      if (k < 0 || LY.blk[k].ic != b.ic) continue;
      const Layout::Blk& yb = LY.blk[k];
      (*yw)[k] = 1;
      TgOut o{};
      o.C = Y + yb.off;
      o.c_f32 = 1;
      o.accumulate = 0;
      TgChunk c{};
      c.A = x_f32 ? (const void*)((const float*)X + b.off) : (const void*)((const double*)X + b.off);
      c.a_f32 = x_f32 ? 1 : 0;
      c.alpha = 1.0f;
      const long long prow = S.offset(dst), pcol = S.offset(src);
      c.B = op.ptr + prow * dimP + pcol;   // element (j = output index, k = input index)
      c.bj = dimP;
      c.bk = 1;
      if (leg == 0) {
        // rows (b, c) linear, K = a with stride db dc; out (a', b, c)
        o.rows = b.db * b.dc; o.N = yb.da;
        o.R2 = kTgRowsBig; o.t1 = 0; o.t2 = 1; o.cj = (long long)yb.db * yb.dc;
        c.R2 = kTgRowsBig; c.s1 = 0; c.s2 = 1; c.sk = (long long)b.db * b.dc; c.K = b.da;
      } else {
        // rows (a, c), K = b with stride dc; out (a, b', c)
        o.rows = b.da * b.dc; o.N = yb.db;
        o.R2 = b.dc; o.t1 = (long long)yb.db * yb.dc; o.t2 = 1; o.cj = yb.dc;
        c.R2 = b.dc; c.s1 = (long long)b.db * b.dc; c.s2 = 1; c.sk = b.dc; c.K = b.db;
      }
      o.npad = (o.N + 15) / 16 * 16;
      pl.max_npad = std::max(pl.max_npad, o.npad);
      o.n_parts = (int)pl.chunks.size();   // chunk_begin while building
      pl.chunks.push_back(c);
      pl.flops += 2.0 * o.rows * o.N * c.K;
      pl.outs.push_back(o);
      tg_tiles(pl, (int)pl.outs.size() - 1, 1);
    }
  };
  struct Src { const void* Z; bool f32; int shift; std::vector<char> written; };
  std::vector<Src> srcs;
  float* zp = tg_pool_;
  for (const HTerm& h : hts) {
    Src sr{x_in_, false, 0, {}};
    if (h.op[0].kind && h.op[1].kind) {
      const int s0 = h.op[0].shift, s1 = h.op[1].shift;
      std::vector<char> w1(lays[s0].blk.size(), 0), w2(lays[s0 + s1].blk.size(), 0);
      leg_apply(T.st[0], L, x_in_, false, nullptr, lays[s0], zp, &w1, 0, h.op[0], s0, d0);
      leg_apply(T.st[1], lays[s0], zp, true, &w1, lays[s0 + s1], zp + zsize, &w2, 1, h.op[1], s1, d1);
      sr = Src{zp + zsize, true, s0 + s1, w2};
      zp += 2 * zsize;
    } else if (h.op[0].kind || h.op[1].kind) {
      const int leg = h.op[0].kind ? 0 : 1;
      const int sh = h.op[leg].shift;
      std::vector<char> w(lays[sh].blk.size(), 0);
      leg_apply(T.st[0], L, x_in_, false, nullptr, lays[sh], zp, &w, leg, h.op[leg], sh, leg == 0 ? d0 : d1);
      sr = Src{zp, true, sh, w};
      zp += zsize;
    }
    srcs.push_back(std::move(sr));
  }
  // stage 2: one output per block of y, chunks over terms
  TgPlan& s3 = T.st[2];
  const double cst = constant_;
  int base_tiles = 0;
  for (const Layout::Blk& yb : L.blk) base_tiles += (yb.da * yb.db + 127) / 128;
  const int parts_wanted = std::max(1, std::min(16, (4 * 152) / std::max(1, base_tiles)));
  for (const Layout::Blk& yb : L.blk) {
    TgOut o{};
    o.C = y_out_ + yb.off;
    o.c_f32 = 0;
    o.accumulate = 0;
    o.rows = yb.da * yb.db;
    o.N = yb.dc;
    o.npad = (o.N + 15) / 16 * 16;
    o.R2 = kTgRowsBig; o.t1 = 0; o.t2 = yb.dc; o.cj = 1;
    s3.max_npad = std::max(s3.max_npad, o.npad);
    o.n_parts = (int)s3.chunks.size();
    auto add = [&](const void* Z, bool f32, long long zoff, int dcz, const double* B, long long bj, long long bk,
                   double alpha, bool identity) {
      TgChunk c{};
      c.A = f32 ? (const void*)((const float*)Z + zoff) : (const void*)((const double*)Z + zoff);
      c.a_f32 = f32 ? 1 : 0;
      c.R2 = kTgRowsBig; c.s1 = 0; c.s2 = dcz; c.sk = 1; c.K = dcz;
      c.B = B; c.bj = bj; c.bk = bk;
      c.alpha = (float)alpha;
      s3.chunks.push_back(c);
      if (!identity) s3.flops += 2.0 * o.rows * o.N * dcz;
    };
    if (cst != 0.0) add(x_in_, false, yb.off, yb.dc, ident_, ident_dim_, 1, cst, true);
    for (size_t t = 0; t < hts.size(); ++t) {
      const HTerm& h = hts[t];
      const Layout& LZ = lays[srcs[t].shift];
      const int k = LZ.find(yb.ia, yb.ib);
      if (k < 0) continue;
      if (!srcs[t].written.empty() && !srcs[t].written[k]) continue;
      const Layout::Blk& zb = LZ.blk[k];
      if (h.op[2].kind == 1) {
        if (L.leg[2].find(L.leg[2].q[zb.ic] + h.op[2].shift) != yb.ic) continue;
        add(srcs[t].Z, srcs[t].f32, zb.off, zb.dc,
            h.op[2].ptr + (long long)L.leg[2].offset(yb.ic) * d2 + L.leg[2].offset(zb.ic), d2, 1, h.coef, false);
      } else {
        if (zb.ic != yb.ic) continue;
        add(srcs[t].Z, srcs[t].f32, zb.off, zb.dc, ident_, ident_dim_, 1, h.coef, true);
      }
    }
    s3.outs.push_back(o);
    tg_tiles(s3, (int)s3.outs.size() - 1, parts_wanted);
  }
  long long scratch = 0;
  for (int i = 0; i < 3; ++i) {
    T.st[i].upload(stream_);
    scratch = std::max(scratch, T.st[i].scratch_need);
    T.flops += T.st[i].flops;
  }
  if (scratch > tg_scratch_elems_) {
    if (tg_scratch_) { untrack(tg_scratch_); cudaFree(tg_scratch_); }
    tg_scratch_elems_ = scratch + scratch / 4;
    device_alloc((void**)&tg_scratch_, tg_scratch_elems_ * sizeof(float), "tensor-core partial sums");
    track(tg_scratch_, tg_scratch_elems_ * sizeof(float));
  }
  if (!check(cudaGetLastError(), "tensor-core plan")) return nullptr;
  TgHeff* raw = tp.get();
  tg_cache_[node] = std::move(tp);
  return raw;
}

int Engine::apply_heff_tg() {
  TgHeff* T = tg_plans(center_);
  if (!T) return -1;
  const int elem = precision_ == PREC_BF16 ? 2 : 4;
  const int split = precision_ == PREC_TF32X3 ? 1 : 0;
  cudaEvent_t e0 = nullptr;
  if (profiling_) ev_begin(&e0);
  for (int i = 0; i < 3; ++i) {
    TgPlan& pl = T->st[i];
    const int rc = launch_tg_gemm(elem, split, pl.d_tiles, (int)pl.tiles.size(), pl.d_outs, pl.d_chunks, pl.max_npad,
                                  tg_scratch_, pl.d_red, (int)pl.red.size(), d_err_, stream_, wait_polls);
    if (rc) {
      err_ = "tensor-core contraction: output width outside the supported range";
      return rc;
    }
  }
  if (profiling_) ev_end(e0, KC_HEFF_SIMT_UPPER, T->flops, T->flops, 0.0);
  return check(cudaGetLastError(), "tensor-core contraction") ? 0 : -3;
}

// ------------------------------------------------------------------ profiling
cudaEvent_t Engine::ev_get() {
  if (!ev_pool_.empty()) {
    cudaEvent_t e = ev_pool_.back();
    ev_pool_.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

void Engine::ev_begin(cudaEvent_t* e) {
  *e = ev_get();
  cudaEventRecord(*e, stream_);
}

void Engine::ev_end(cudaEvent_t a, int cls, double fa, double fe, double ba) {
  cudaEvent_t b = ev_get();
  cudaEventRecord(b, stream_);
  ev_pending_.push_back({a, b, cls, fa, fe, ba});
  if (ev_pending_.size() > 4096) {
    KernelTiming dummy[KC_COUNT];
    kernel_timing(dummy);
  }
}

void Engine::set_profiling(bool on) { profiling_ = on; }

void Engine::reset_timing() {
  KernelTiming dummy[KC_COUNT];
  kernel_timing(dummy);
  for (auto& t : timing_) t = KernelTiming();
}

int Engine::kernel_timing(KernelTiming out[KC_COUNT]) {
  if (!check(cudaStreamSynchronize(stream_), "timing")) return -3;
  for (auto& r : ev_pending_) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    KernelTiming& t = timing_[r.cls];
    t.ms += ms;
    t.launches += 1;
    t.flops_alg += r.fa;
    t.flops_exec += r.fe;
    t.bytes_alg += r.ba;
    ev_pool_.push_back(r.a);
    ev_pool_.push_back(r.b);
  }
  ev_pending_.clear();
  for (int i = 0; i < KC_COUNT; ++i) out[i] = timing_[i];
  return 0;
}

// ------------------------------------------------------------------ Lanczos
// Symmetric Lanczos with full reorthogonalisation (classical Gram-Schmidt,
// a second pass when the first removed more than half of the norm), started
// from the current tensor; the lowest Ritz pair of the tridiagonal is found
// on the device.  Stops when the residual estimate |beta_k s_k| <= tol
// |theta|; when the Krylov space is full, a thick restart keeps the lowest
// Ritz vectors.
int Engine::lanczos(int node, double tol, int max_krylov, bool mixed, int max_restarts, double* energy, double* resid,
                    int* iters) {
  cudaEvent_t e0 = nullptr;
  if (profiling_) ev_begin(&e0);
  int rc = lanczos_run(node, tol, max_krylov, mixed, max_restarts, energy, resid, iters);
  if (profiling_) ev_end(e0, KC_LANCZOS, 0, 0, 0);
  return rc;
}

// ---- Lanczos building blocks (shared by the single-state and the batched
// drivers).  Scalars live in d_scal_: alpha[128], beta[128], s[128], out,
// Gram-Schmidt coefficients, norms; a thick restart's k x keep combination.
namespace {
constexpr int kAlpha = 0, kBeta = 128, kSvec = 256, kOut = 384, kCoef = 512, kNrm2 = 640, kNrmPre = 641,
              kNrmMid = 642, kCmat = 1024, kC1 = 2048, kC2 = 2304, kMid = 2500, kNrmSecond = 2501;
}

int Engine::lz_prepare(int kmax) {
  if (kmax_alloc_ < kmax + 1) {
    if (V_) { untrack(V_); cudaFree(V_); }
    if (!check(cudaMalloc(&V_, (size_t)(kmax + 1) * nmax_ * sizeof(double)), "Krylov basis")) return -2;
    track(V_, (size_t)(kmax + 1) * nmax_ * sizeof(double));
    kmax_alloc_ = kmax + 1;
  }
  const int keep = std::min(kThickKeep, kmax / 4);
  if (keep >= 1 && zb_elems_ < (long long)keep * nmax_) {
    if (zb_) { untrack(zb_); cudaFree(zb_); }
    zb_elems_ = (long long)keep * nmax_;
    if (!check(cudaMalloc(&zb_, zb_elems_ * sizeof(double)), "restart basis")) return -2;
    track(zb_, zb_elems_ * sizeof(double));
  }
  return 0;
}

// v_0 = T[node] / |T[node]|
void Engine::lz_start(int node) {
  const long long n = layout_[node].size;
  launch_copy(T_[node], tmp_, n, stream_);
  launch_dot(tmp_, tmp_, n, d_partial_, d_scal_ + kNrm2, stream_);
  launch_scale_inv_sqrt(tmp_, V_, n, d_scal_ + kNrm2, stream_);
}

// With y_out_ = H_eff v_j: alpha_j, the three-term recurrence folded into the
// first classical Gram-Schmidt pass against all j + 1 basis vectors (the
// coefficients come from the reduced vector, as in a separate three-term
// step, so that rounding stays relative to beta_j and not to alpha_j), a
// second pass only if the first removed more than half of ||w'||^2 (Daniel-
// Gragg-Kaufman-Stewart, decided on the device), beta_j = ||w|| and
// v_{j+1} = w / beta_j (column kmax holds the residual vector of a full
// cycle).  Eleven launches.
void Engine::lz_iteration(int j, long long n) {
  launch_lz_reorth(V_, nmax_, j + 1, y_out_, n, d_partial_, d_scal_ + kC1, d_scal_ + kC2, d_scal_ + kMid,
                   d_scal_ + kNrmSecond, kReorthRatio, d_scal_ + kAlpha + j, j > 0 ? d_scal_ + kBeta + j - 1 : nullptr,
                   d_scal_ + kBeta + j, d_scal_ + kNrm2, V_ + (long long)(j + 1) * nmax_, stream_,
                   precision_ != PREC_FP64 ? 1 : 0);
}

// v_{j+1} is written by lz_iteration.
void Engine::lz_next_vector(int j, long long n) {
  (void)j;
  (void)n;
}

// Thick restart after a full cycle of k vectors (see lanczos_restart_kernel);
// *j0 = vectors carried into the next cycle.  Synchronises the stream.
int Engine::lz_thick_restart(int k, int kmax, long long n, int* j0) {
  const long long ld = nmax_;
  double* alpha = d_scal_ + kAlpha;
  double* beta = d_scal_ + kBeta;
  const int keep = std::min(kThickKeep, kmax / 4);
  if (keep < 1) {   // explicit restart from the Ritz vector
    launch_tridiag_lowest(alpha, beta, k, d_scal_ + kOut, d_scal_ + kSvec, 1, stream_);
    launch_combine(V_, ld, k, d_scal_ + kSvec, tmp_, n, stream_);
    launch_dot(tmp_, tmp_, n, d_partial_, d_scal_ + kNrm2, stream_);
    launch_scale_inv_sqrt(tmp_, V_, n, d_scal_ + kNrm2, stream_);
    *j0 = 0;
    return 0;
  }
  launch_lanczos_restart(alpha, beta, k, keep, d_scal_ + kCmat, d_err_ + 1, stream_);
  int p = 0;
  cudaMemcpyAsync(&p, d_err_ + 1, sizeof(int), cudaMemcpyDeviceToHost, stream_);
  if (!check(cudaStreamSynchronize(stream_), "thick restart")) return -3;
  if (p < 1 || p > keep) {
    err_ = "thick restart: invalid kept count";
    return -3;
  }
  launch_rotate_basis(V_, ld, k, d_scal_ + kCmat, p, zb_, n, stream_);
  cudaMemcpyAsync(V_, zb_, (size_t)p * ld * sizeof(double), cudaMemcpyDeviceToDevice, stream_);
  launch_copy(V_ + (long long)kmax * ld, V_ + (long long)p * ld, n, stream_);
  *j0 = p;
  return 0;
}

// Ritz vector x = V s of the last k vectors, normalised into T[node]; the
// Ritz value and residual estimate go to the final ring slot (read after a
// synchronisation).
void Engine::lz_finish(int node, int k) {
  const long long n = layout_[node].size;
  launch_tridiag_lowest(d_scal_ + kAlpha, d_scal_ + kBeta, k, d_scal_ + kOut, d_scal_ + kSvec, 1, stream_);
  launch_combine(V_, nmax_, k, d_scal_ + kSvec, tmp_, n, stream_);
  launch_dot(tmp_, tmp_, n, d_partial_, d_scal_ + kNrm2, stream_);
  launch_scale_inv_sqrt(tmp_, T_[node], n, d_scal_ + kNrm2, stream_);
  cudaMemcpyAsync(ring_host_ + 4 * kMaxKrylov, d_scal_ + kOut, 2 * sizeof(double), cudaMemcpyDeviceToHost, stream_);
}

// Convergence data of iteration j (lowest Ritz pair of T_{j+1}, beta_j) into
// ring slot j, computed on the side stream.
void Engine::lz_queue_check(int j) {
  cudaEventRecord(ev_iter_[j], stream_);
  cudaStreamWaitEvent(aux_, ev_iter_[j], 0);
  launch_tridiag_lowest(d_scal_ + kAlpha, d_scal_ + kBeta, j + 1, ring_dev_ + 4 * j, d_scal_ + kSvec, 0, aux_);
  cudaMemcpyAsync(ring_host_ + 4 * j, ring_dev_ + 4 * j, 2 * sizeof(double), cudaMemcpyDeviceToHost, aux_);
  cudaMemcpyAsync(ring_host_ + 4 * j + 2, d_scal_ + kBeta + j, sizeof(double), cudaMemcpyDeviceToHost, aux_);
  cudaEventRecord(ev_conv_[j], aux_);
  last_conv_ = j;
}

bool Engine::lz_converged(int slot, double tol, double* theta, double* res) const {
  const double* h = ring_host_ + 4 * slot;
  *theta = h[0];
  *res = h[1];
  const bool breakdown = h[2] <= 1e-13 * std::max(1.0, std::fabs(*theta));
  return *res <= tol * std::max(1e-300, std::fabs(*theta)) || breakdown;
}

int Engine::lanczos_run(int node, double tol, int max_krylov, bool mixed, int max_restarts, double* energy,
                        double* resid, int* iters) {
  use_mixed_ = mixed;
  const long long n = layout_[node].size;
  int kmax = std::min(std::max(max_krylov, 2), kMaxKrylov);
  if (kmax > n) kmax = (int)n;
  int rc = lz_prepare(kmax);
  if (rc) return rc;
  lz_start(node);
  int total_iters = 0;
  double theta = 0.0, res = 0.0, prev_res = 1e300;
  int stalls = 0;
  int j0 = 0;   // vectors carried into the cycle (thick restart)
  int k = 0;
  // no speculation in the FP64 check of a mixed state: it usually ends
  // after one product, and a speculative one would be a wasted FP64 product
  const bool speculate = mixed || precision_ == PREC_FP64;
  for (int restart = 0; restart < max_restarts; ++restart) {
    if (restart > 0 && (rc = lz_thick_restart(k, kmax, n, &j0))) return rc;
    // The convergence data of iteration j is computed on a side stream and
    // read one iteration later, so the host never waits with an empty GPU
    // queue: iteration j+1 is already queued (speculatively) when iteration
    // j is found converged; it only writes alpha/beta/V entries past the
    // converged basis.
    bool done = false;
    int pending = -1;
    for (int j = j0; j < kmax; ++j) {
      if ((rc = apply_heff(V_ + j * nmax_, y_out_, -1))) return rc;
      ++total_iters;
      lz_iteration(j, n);
      lz_queue_check(j);
      lz_next_vector(j, n);
      k = j + 1;
      if (!speculate) {
        if (!check(cudaEventSynchronize(ev_conv_[j]), "lanczos")) return -3;
        if (lz_converged(j, tol, &theta, &res)) { done = true; break; }
        continue;
      }
      if (pending >= 0) {
        if (!check(cudaEventSynchronize(ev_conv_[pending]), "lanczos")) return -3;
        if (lz_converged(pending, tol, &theta, &res)) { k = pending + 1; done = true; break; }
      }
      pending = j;
    }
    if (!done && pending >= 0) {
      if (!check(cudaEventSynchronize(ev_conv_[pending]), "lanczos")) return -3;
      k = pending + 1;
      done = lz_converged(pending, tol, &theta, &res);
    }
    if (done) break;
    // a low-precision operator stops improving at its rounding level: two
    // restart cycles within 1000x of that level without a 2 % gain end the
    // low-precision phase
    if (mixed) {
      const bool near_floor = res <= 1e3 * mixed_tol * std::fabs(theta);
      stalls = (near_floor && res > 0.98 * prev_res) ? stalls + 1 : 0;
      if (stalls >= 2) break;
    }
    prev_res = std::min(prev_res, res);
  }
  lz_finish(node, k);
  use_mixed_ = false;
  if (!check(cudaStreamSynchronize(stream_), "lanczos end")) return -3;
  // a speculative iteration's convergence data may still be in flight
  if (last_conv_ >= 0 && !check(cudaEventSynchronize(ev_conv_[last_conv_]), "lanczos end")) return -3;
  last_conv_ = -1;
  *energy = ring_host_[4 * kMaxKrylov];
  *resid = ring_host_[4 * kMaxKrylov + 1];
  *iters = total_iters;
  return 0;
}

// Node update.  FP64 path: Lanczos to tol.  Mixed path (bottom nodes):
// Lanczos with tensor-core matvecs to max(tol, mixed_tol), then the same
// Lanczos restarted from that Ritz vector with FP64 matvecs until the FP64
// residual meets tol (the FP64 residual correction).
int Engine::optimize_node(int node, double tol, int max_krylov, SweepStats* st, double* e) {
  int rc = move_to(node);
  if (rc) return rc;
  double energy = 0, res = 0;
  int iters = 0, mixed_iters = 0;
  last_mixed_ritz = std::nan("");
  last_mixed_residual = std::nan("");
  if (mixed_node(node)) {
    cudaMemsetAsync(d_err_, 0, sizeof(int), stream_);
    // the low-precision phase aims a little below tol so that the FP64
    // check usually passes on its first product
    rc = lanczos(node, std::max(0.3 * tol, mixed_tol), max_krylov, true, 50, &energy, &res, &mixed_iters);
    if (rc) return rc;
    last_mixed_ritz = energy;
    last_mixed_residual = res / std::max(1e-300, std::fabs(energy));
    int herr = 0;
    cudaMemcpyAsync(&herr, d_err_, sizeof(int), cudaMemcpyDeviceToHost, stream_);
    if (!check(cudaStreamSynchronize(stream_), "mixed phase")) return -3;
    if (herr) {
      err_ = "tensor-core H_eff: an mbarrier wait hit its iteration limit";
      return -6;
    }
  }
  // the FP64 residual correction: float-float products in a mixed state
  ff_products_ = mixed_node(node);
  rc = lanczos(node, tol, max_krylov, false, 50, &energy, &res, &iters);
  ff_products_ = false;
  if (rc) return rc;
  last_lanczos_iters = iters;
  last_mixed_iters = mixed_iters;
  last_residual = res / std::max(1e-300, std::fabs(energy));
  if (st) {
    st->matvecs += iters + mixed_iters;
    st->matvecs_mixed += mixed_iters;
    st->node_updates += 1;
    st->energy = energy;
    st->max_residual = std::max(st->max_residual, res / std::max(1e-300, std::fabs(energy)));
    if (res > tol * std::fabs(energy)) st->not_converged += 1;
  }
  if (e) *e = energy;
  return 0;
}

int Engine::sweep(double tol, int max_krylov, SweepStats* st, std::vector<double>* energies) {
  for (int i : sweep_order(nodes_)) {
    double e = 0;
    int rc = optimize_node(i, tol, max_krylov, st, &e);
    if (rc) return rc;
    if (energies) energies->push_back(e);
  }
  return 0;
}

// ------------------------------------------------------------------ measurement
int Engine::energy(double* total, double parts[N_CLASSES]) {
  const long long n = layout_[center_].size;
  double* nrm2 = d_scal_ + 640;
  double* dv = d_scal_ + 700;
  launch_dot(T_[center_], T_[center_], n, d_partial_, nrm2, stream_);
  int rc = apply_heff(T_[center_], tmp_, -1);
  if (rc) return rc;
  launch_dot(T_[center_], tmp_, n, d_partial_, dv, stream_);
  for (int c = 0; c < N_CLASSES; ++c) {
    rc = apply_heff(T_[center_], tmp_, c);
    if (rc) return rc;
    launch_dot(T_[center_], tmp_, n, d_partial_, dv + 1 + c, stream_);
  }
  double host[2 + N_CLASSES];
  cudaMemcpyAsync(host, nrm2, sizeof(double), cudaMemcpyDeviceToHost, stream_);
  cudaMemcpyAsync(host + 1, dv, (1 + N_CLASSES) * sizeof(double), cudaMemcpyDeviceToHost, stream_);
  if (!check(cudaStreamSynchronize(stream_), "energy")) return -3;
  *total = host[1] / host[0];
  for (int c = 0; c < N_CLASSES; ++c) parts[c] = host[2 + c] / host[0];
  return 0;
}

// Reduced density matrices pushed down from the root: rho_child[i', i] =
// sum T[.., i', .., c'] rho[c', c] T[.., i, .., c].  Returns the 267
// diagonal entries per site.
int Engine::site_probabilities(std::vector<double>* probs) {
  int rc = move_to((int)nodes_.size() - 1);
  if (rc) return rc;
  const int n = (int)nodes_.size();
  std::vector<double*> rho(n, nullptr);
  probs->assign((size_t)lat_.n_sites() * kLocalDim, 0.0);
  double* one = nullptr;
  device_alloc((void**)&one, sizeof(double), "density matrix");
  track(one, sizeof(double));
  const double v1 = 1.0;
  cudaMemcpyAsync(one, &v1, sizeof(double), cudaMemcpyHostToDevice, stream_);
  rho[n - 1] = one;
  std::vector<void*> tofree{one};
  for (int idx = n - 1; idx >= 0 && rc == 0; --idx) {
    const Layout& L = layout_[idx];
    const int dp = L.leg[2].total();
    // Y = rho (x)_2 T  (rho symmetric)
    cudaMemsetAsync(tmp_, 0, L.size * sizeof(double), stream_);
    work_.clear();
    plan_leg_apply(work_, L, T_[idx], L, tmp_, 2, rho[idx], dp, 0, false, 1.0);
    rc = run_plan(work_);
    for (int leg = 0; leg < 2 && rc == 0; ++leg) {
      const int d = L.leg[leg].total();
      double* red = nullptr;
      device_alloc((void**)&red, (size_t)d * d * sizeof(double), "density matrix");
      track(red, (size_t)d * d * sizeof(double));
      tofree.push_back(red);
      cudaMemsetAsync(red, 0, (size_t)d * d * sizeof(double), stream_);
      work_.clear();
      plan_contract_but(work_, L, T_[idx], L, tmp_, leg, red, d, 1.0);
      rc = run_plan(work_);
      if (nodes_[idx].child_kind[leg] == 1) {
        rho[nodes_[idx].child[leg]] = red;
      } else {
        std::vector<double> h((size_t)d * d);
        cudaMemcpyAsync(h.data(), red, h.size() * sizeof(double), cudaMemcpyDeviceToHost, stream_);
        cudaStreamSynchronize(stream_);
        const int s = nodes_[idx].child[leg];
        for (int a = 0; a < kLocalDim; ++a) (*probs)[(size_t)s * kLocalDim + a] = h[(size_t)a * d + a];
      }
    }
  }
  cudaStreamSynchronize(stream_);
  for (void* p : tofree) { untrack(p); cudaFree(p); }
  return rc ? rc : (check(cudaGetLastError(), "probabilities") ? 0 : -3);
}

int Engine::node_export(int node, std::vector<double>* host) {
  host->resize(layout_[node].size);
  cudaMemcpyAsync(host->data(), T_[node], host->size() * sizeof(double), cudaMemcpyDeviceToHost, stream_);
  return check(cudaStreamSynchronize(stream_), "export") ? 0 : -3;
}

int Engine::node_import(int node, const std::vector<double>& host) {
  if ((long long)host.size() != layout_[node].size) return -1;
  for (double v : host)
    if (!std::isfinite(v)) return -5;
  cudaMemcpyAsync(T_[node], host.data(), host.size() * sizeof(double), cudaMemcpyHostToDevice, stream_);
  return check(cudaStreamSynchronize(stream_), "import") ? 0 : -3;
}

int Engine::load_tensors(const double* const* host, const long long* sizes, int n) {
  if (n != (int)nodes_.size()) return -1;
  for (int i = 0; i < n; ++i)
    if (sizes[i] != layout_[i].size || !host[i]) return -1;
  for (int i = 0; i < n; ++i)
    cudaMemcpyAsync(T_[i], host[i], sizes[i] * sizeof(double), cudaMemcpyHostToDevice, stream_);
  // non-finite entries are looked for on the device, after the copies
  cudaMemsetAsync(d_err_ + 2, 0, sizeof(int), stream_);
  for (int i = 0; i < n; ++i) launch_check_finite(T_[i], sizes[i], d_err_ + 2, stream_);
  int bad = 0;
  cudaMemcpyAsync(&bad, d_err_ + 2, sizeof(int), cudaMemcpyDeviceToHost, stream_);
  if (!check(cudaStreamSynchronize(stream_), "load")) return -3;
  if (bad) {
    err_ = "non-finite tensor entry";
    return -5;
  }
  tc_w_node_ = -1;
  for (const TreeNode& nd : nodes_)
    if (nd.parent >= 0) {
      int rc = compute_up(nd.index);
      if (rc) return rc;
    }
  center_ = (int)nodes_.size() - 1;
  return check(cudaGetLastError(), "load") ? 0 : -3;
}

int Engine::set_couplings(const Params& np) {
  if (np.Lx != p_.Lx || np.Ly != p_.Ly || np.Lz != p_.Lz || np.boundary != p_.boundary || np.Q != p_.Q) {
    err_ = "set_couplings: the lattice, the boundary and the charge sector are fixed";
    return -1;
  }
  const double oldc[N_COUPLINGS] = {p_.t, p_.m, p_.ge2, p_.cB, p_.nu};
  const double newc[N_COUPLINGS] = {np.t, np.m, np.ge2, np.cB, np.nu};
  for (int c = 0; c < N_COUPLINGS; ++c)
    if (!std::isfinite(newc[c]) || (oldc[c] == 0.0 && newc[c] != 0.0)) {
      err_ = "set_couplings: a coupling is not finite, or its class was zero at creation (no terms)";
      return -1;
    }
  // same term list as a fresh model with these couplings; a class switched
  // off keeps its terms with coefficient zero
  Params sub = np;
  sub.mu = p_.mu;   // the chemical potentials stay as created
  double* subc[N_COUPLINGS] = {&sub.t, &sub.m, &sub.ge2, &sub.cB, &sub.nu};
  for (int c = 0; c < N_COUPLINGS; ++c)
    if (newc[c] == 0.0 && oldc[c] != 0.0) *subc[c] = 1.0;
  std::vector<Term> nt;
  double cst = 0.0;
  build_terms(sub, &nt, &cst);
  if (nt.size() != terms_.size()) {
    err_ = "set_couplings: term list changed";
    return -1;
  }
  for (size_t i = 0; i < nt.size(); ++i)
    if (nt[i].cls != terms_[i].cls || nt[i].ops.size() != terms_[i].ops.size()) {
      err_ = "set_couplings: term list changed";
      return -1;
    }
  for (size_t i = 0; i < nt.size(); ++i)
    terms_[i].coef = (nt[i].cls < N_COUPLINGS && newc[nt[i].cls] == 0.0) ? 0.0 : nt[i].coef;
  constant_ = cst;
  p_.t = np.t; p_.m = np.m; p_.ge2 = np.ge2; p_.cB = np.cB; p_.nu = np.nu;
  // drop everything that holds a coefficient
  clear_plan_caches();
  clear_tc_cache();
  tg_cache_.clear();
  std::vector<void*> dead;
  for (auto& kv : oz_cache_)
    for (void* p : kv.second->owned) dead.push_back(p);
  oz_cache_.clear();
  for (auto it = rowmaps_.begin(); it != rowmaps_.end();) {
    if (it->first.second <= -1000) {   // site Hamiltonian maps (coefficients in their values)
      for (RowMap& rm : it->second) {
        dead.push_back(rm.map);
        dead.push_back(rm.val);
      }
      it = rowmaps_.erase(it);
    } else {
      ++it;
    }
  }
  for (auto& kv : inv_maps_) {
    dead.push_back(kv.second.map);
    dead.push_back(kv.second.val);
  }
  inv_maps_.clear();
  dfree_all(dead);
  ++gen_;
  tc_w_node_ = -1;
  for (const TreeNode& nd : nodes_)
    if (nd.parent >= 0) {
      int rc = compute_up(nd.index);
      if (rc) return rc;
    }
  center_ = (int)nodes_.size() - 1;
  return check(cudaGetLastError(), "set_couplings") ? 0 : -3;
}

int Engine::noalloc_worklist(const double* x, double* y, KTile* tiles, int max_tiles, KOutput* outs, int max_outs,
                             KChunk* chunks, int max_chunks, int* n_tiles, int* n_outs, int* n_chunks) {
  const int node = center_;
  const TreeNode& nd = nodes_[node];
  if (nd.child_kind[0] != 0 || nd.child_kind[1] != 0) {
    err_ = "the centre is not a bottom node";
    return -7;
  }
  const Layout& L = layout_[node];
  const Sectors& P = L.leg[2];
  const int d2 = P.total();
  const bool root = nd.parent < 0;
  const int sl = nd.child[0], sr = nd.child[1];
  int no = 0, nc = 0, nt = 0;
  auto find_maps = [&](int key) -> const std::vector<RowMap>* {
    auto it = rowmaps_.find(std::make_pair(node, key));
    return it == rowmaps_.end() ? nullptr : &it->second;
  };
  for (size_t oc = 0; oc < P.q.size(); ++oc) {
    const int rows = L.sec_rows[oc];
    if (rows == 0) continue;
    const int dc = P.dim[oc];
    if (no >= max_outs) { err_ = "work list: too many outputs"; return -2; }
    KOutput& o = outs[no];
    o.C = y + L.sec_off[oc];
    o.c_m = dc;
    o.c_n = 1;
    o.M = rows;
    o.N = dc;
    o.chunk_begin = nc;
    o.accumulate = 0;
    o.n_parts = 1;
    o.part_off = 0;
    auto push = [&](const KChunk& c) -> bool {
      if (nc >= max_chunks) return false;
      chunks[nc++] = c;
      return true;
    };
    if (constant_ != 0.0) {
      KChunk c = make_chunk();
      c.A = x + L.sec_off[oc]; c.a_m = dc; c.a_k = 1; c.add = 1; c.alpha = constant_;
      if (!push(c)) { err_ = "work list: too many chunks"; return -2; }
    }
    // single-site terms of both sites: the all-class diagonal if present,
    // otherwise one map per coupling class
    for (int leg = 0; leg < 2; ++leg) {
      const std::vector<RowMap>* all = find_maps(-1000 - 10 * leg);
      for (int cls = all ? -1 : 0; cls < (all ? 0 : N_CLASSES); ++cls) {
        const std::vector<RowMap>* maps = find_maps(-1000 - 10 * leg - (cls + 1));
        if (!maps) { err_ = "site map missing at this centre"; return -7; }
        const RowMap& rm = (*maps)[oc];
        if (rm.src_sector < 0) continue;
        KChunk c = make_chunk();
        c.A = x + L.sec_off[rm.src_sector]; c.a_m = P.dim[rm.src_sector]; c.a_k = 1;
        c.amap = rm.map; c.aval = rm.val; c.add = 1;
        if (!push(c)) { err_ = "work list: too many chunks"; return -2; }
      }
    }
    if (!root) {
      KChunk c = make_chunk();
      c.A = x + L.sec_off[oc]; c.a_m = dc; c.a_k = 1;
      c.B = down_[node].Htot + P.offset((int)oc) * (long long)d2 + P.offset((int)oc); c.b_k = 1; c.b_n = d2;
      c.K = dc;
      if (!push(c)) { err_ = "work list: too many chunks"; return -2; }
    }
    for (int k = 0; k < (int)terms_.size(); ++k) {
      bool t[3] = {false, false, false};
      for (auto& so : terms_[k].ops) {
        if (so.first == sl) t[0] = true;
        else if (so.first == sr) t[1] = true;
        else t[2] = true;
      }
      if ((int)t[0] + (int)t[1] + (int)t[2] < 2) continue;
      const std::vector<RowMap>* maps = find_maps(k);
      if (!maps) { err_ = "row map missing at this centre"; return -7; }
      const RowMap& rm = (*maps)[oc];
      if (rm.src_sector < 0) continue;
      const int ic = rm.src_sector;
      KChunk c = make_chunk();
      c.A = x + L.sec_off[ic]; c.a_m = P.dim[ic]; c.a_k = 1;
      c.amap = rm.map; c.aval = rm.val; c.alpha = terms_[k].coef;
      if (t[2]) {
        auto it = down_[node].term.find(k);
        if (it == down_[node].term.end()) { err_ = "environment operator missing"; return -7; }
        if (P.find(P.q[ic] + it->second.shift) != (int)oc) continue;
        c.B = it->second.ptr + P.offset((int)oc) * (long long)d2 + P.offset(ic); c.b_k = 1; c.b_n = d2;
        c.K = P.dim[ic];
      } else {
        if (ic != (int)oc) continue;
        c.add = 1;
      }
      if (!push(c)) { err_ = "work list: too many chunks"; return -2; }
    }
    o.chunk_end = nc;
    for (int m0 = 0; m0 < rows; m0 += KT_BM)
      for (int n0 = 0; n0 < dc; n0 += KT_BN) {
        if (nt >= max_tiles) { err_ = "work list: too many tiles"; return -2; }
        tiles[nt++] = KTile{no, m0, n0, o.chunk_begin, o.chunk_end, -1};
      }
    ++no;
  }
  *n_tiles = nt;
  *n_outs = no;
  *n_chunks = nc;
  return 0;
}

}  // namespace qed
