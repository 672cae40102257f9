// Batched sweeps of independent TTN problems (same lattice, same precision,
// one CUDA stream).  The problems update the same node together: centre
// moves per problem, then one lockstep Lanczos whose H_eff products for
// all problems are a single grouped launch (tensor-core tiles of every
// problem's bottom-node plan, or every problem's grouped-GEMM chunks above),
// replayed from a CUDA graph once its tile shapes are tuned (upper nodes of a
// mixed batch: every problem's tensor-core stage plans).  The vector
// work of each problem follows on the same stream, and one wait per lockstep
// iteration reads every problem's convergence data.  The FP64 check of a
// mixed-precision update runs per problem afterwards.  Every problem does
// the same arithmetic as an unbatched sweep, product tiles included, except
// that the grouped GEMM of a batch is tuned and split on the whole batch.
#include <algorithm>
#include <cmath>
#include <map>
#include <memory>
#include <stdexcept>

#include "batch.h"
#include "engine.h"

namespace qed {

namespace {
constexpr double kRebuildFraction = 0.75;   // new grouped plan when fewer members stay active
}

struct BatchRunner::Grouped {
  std::vector<int> members;
  std::vector<uint64_t> gens;   // members' plan-cache generations at build time
  double* scratch = nullptr;    // launcher's split-K scratch at capture time
  bool tc = false;
  bool tg = false;              // upper node of a mixed batch: tensor-core leg contractions
  bool launched = false;        // one eager launch before any graph capture
  int fp32 = 0;
  TcPlan tcp;
  KPlan st[3];
  TgPlan tgs[3];
  float* tg_scratch = nullptr;
  std::vector<std::pair<double*, long long>> zero;   // Z pools to clear before the stages
  cudaGraphExec_t exec = nullptr;
  long long graph_kernels = 0;
  ~Grouped() {
    if (exec) cudaGraphExecDestroy(exec);
    if (tg_scratch) cudaFree(tg_scratch);
  }
};

// Grouped plans touch every member's memory: the plan validator of each
// engine consults the others' allocations during the batch.
BatchRunner::BatchRunner(std::vector<Engine*> es) : es_(std::move(es)) {
  for (Engine* e : es_) e->peers_.assign(es_.begin(), es_.end());
}

BatchRunner::~BatchRunner() {
  if (!es_.empty()) cudaStreamSynchronize(es_[0]->stream_);
  for (Engine* e : es_) e->peers_.clear();
}

namespace {
template <typename T>
void append(std::vector<T>* dst, const std::vector<T>& src) {
  dst->insert(dst->end(), src.begin(), src.end());
}

template <typename T>
void upload_vec(T*& dptr, size_t& cap, const std::vector<T>& host, cudaStream_t s) {
  if (host.empty()) return;
  if (host.size() > cap) {
    if (dptr) cudaFree(dptr);
    cap = host.size();
    device_alloc((void**)&dptr, cap * sizeof(T), "grouped plan arrays");
  }
  cudaMemcpyAsync(dptr, host.data(), host.size() * sizeof(T), cudaMemcpyHostToDevice, s);
}
}  // namespace

// Concatenation of the members' product plans at the current centre.
int BatchRunner::build(int node, const std::vector<int>& members, std::unique_ptr<Grouped>* out) {
  Engine* e0 = es_[members[0]];
  std::unique_ptr<Grouped> g(new Grouped);
  g->members = members;
  const bool bottom = e0->nodes_[node].child_kind[0] == 0;
  const bool mixed = e0->precision_ != PREC_FP64;
  g->tc = bottom && mixed;
  g->fp32 = mixed ? 1 : 0;
  if (g->tc) {
    TcPlan& b = g->tcp;
    for (int m : members) {
      Engine* e = es_[m];
      TcPlan* t = e->tc_prepare();
      if (!t) return -1;
      const int o0 = (int)b.outs.size(), c0 = (int)b.chunks.size(), a0 = (int)b.adds.size();
      for (TcTile tl : t->tiles) {
        tl.out += o0;
        b.tiles.push_back(tl);
      }
      for (TcOutput o : t->outs) {
        o.chunk_begin += c0;
        o.chunk_end += c0;
        o.add_begin += a0;
        o.add_end += a0;
        b.outs.push_back(o);
      }
      append(&b.chunks, t->chunks);
      append(&b.adds, t->adds);
      append(&b.xjobs, t->xjobs);
      b.x_max_elems = std::max(b.x_max_elems, t->x_max_elems);
      b.max_kpad = std::max(b.max_kpad, t->max_kpad);
      b.max_npad = std::max(b.max_npad, t->max_npad);
      b.flops_alg += t->flops_alg;
      b.flops_exec += t->flops_exec;
      b.bytes_alg += t->bytes_alg;
    }
    cudaStream_t s = e0->stream_;
    upload_vec(b.d_tiles, b.cap[0], b.tiles, s);
    upload_vec(b.d_outs, b.cap[1], b.outs, s);
    upload_vec(b.d_chunks, b.cap[2], b.chunks, s);
    upload_vec(b.d_adds, b.cap[3], b.adds, s);
    upload_vec(b.d_xjobs, b.cap[4], b.xjobs, s);
  } else if (mixed) {
    // upper node, mixed: every member's tensor-core stage plans, concatenated
    // stage by stage; partial sums rebased into one batch scratch
    g->tg = true;
    for (int m : members)
      if (!es_[m]->tg_plans(node)) return -1;
    long long scratch = 0;
    for (int i = 0; i < 3; ++i) {
      TgPlan& b = g->tgs[i];
      long long part_base = 0;
      for (int m : members) {
        const TgPlan& p = es_[m]->tg_plans(node)->st[i];
        const int o0 = (int)b.outs.size(), c0 = (int)b.chunks.size();
        for (TgTile t : p.tiles) {
          t.out += o0;
          t.chunk_begin += c0;
          t.chunk_end += c0;
          b.tiles.push_back(t);
        }
        for (TgOut o : p.outs) {
          if (o.n_parts > 1) o.part_off += part_base;
          b.outs.push_back(o);
        }
        for (int r : p.red) b.red.push_back(r + o0);
        append(&b.chunks, p.chunks);
        part_base += p.scratch_need;
        b.max_npad = std::max(b.max_npad, p.max_npad);
        b.flops += p.flops;
      }
      b.scratch_need = part_base;
      scratch = std::max(scratch, part_base);
      b.upload(e0->stream_);
    }
    device_alloc((void**)&g->tg_scratch, (size_t)std::max(scratch, 1LL) * sizeof(float), "batched partial sums");
  } else {
    for (int m : members) {
      Engine* e = es_[m];
      Engine::HeffPlans* hp = e->heff_plans(node, -1, false);
      if (!hp) return -1;
      if (!bottom && hp->z_elems > 0) g->zero.push_back({e->zpool_, hp->z_elems});
    }
    // (a member's heff_plans may have rebuilt that member's caches: read the
    // plans again now that all exist)
    for (int i = 0; i < 3; ++i) {
      KPlan& b = g->st[i];
      for (int m : members) {
        const KPlan& p = es_[m]->heff_plans(node, -1, false)->st[i];
        const int c0 = (int)b.chunks.size();
        for (KOutput o : p.outs) {
          o.chunk_begin += c0;
          o.chunk_end += c0;
          b.outs.push_back(o);
        }
        append(&b.chunks, p.chunks);
      }
      b.finalize(4096);
    }
  }
  for (int m : members) g->gens.push_back(es_[m]->gen_);
  *out = std::move(g);
  return 0;
}

bool BatchRunner::stale(const Grouped& g) const {
  for (size_t i = 0; i < g.members.size(); ++i)
    if (es_[g.members[i]]->gen_ != g.gens[i]) return true;
  return false;
}

// The launches of one grouped product (eager, or recorded into a graph).
int BatchRunner::launch(Grouped& g) {
  Engine* e0 = es_[g.members[0]];
  cudaStream_t s = e0->stream_;
  if (g.tc) {
    const int elem = e0->precision_ == PREC_BF16 ? 2 : 4;
    const int split = e0->precision_ == PREC_TF32X3 ? 1 : 0;
    launch_convert(elem, split, g.tcp.d_xjobs, (int)g.tcp.xjobs.size(), g.tcp.x_max_elems, s);
    const int rc = launch_tc_heff(elem, split, g.tcp.d_tiles, (int)g.tcp.tiles.size(), g.tcp.d_outs, g.tcp.d_chunks,
                                  g.tcp.d_adds, g.tcp.max_kpad, g.tcp.max_npad, e0->d_err_, s);
    if (rc) e0->err_ = "tensor-core H_eff: tile shape outside the supported range";
    return rc;
  }
  if (g.tg) {
    const int elem = e0->precision_ == PREC_BF16 ? 2 : 4;
    const int split = e0->precision_ == PREC_TF32X3 ? 1 : 0;
    for (int i = 0; i < 3; ++i) {
      TgPlan& p = g.tgs[i];
      const int rc = launch_tg_gemm(elem, split, p.d_tiles, (int)p.tiles.size(), p.d_outs, p.d_chunks, p.max_npad,
                                    g.tg_scratch, p.d_red, (int)p.red.size(), e0->d_err_, s, e0->wait_polls);
      if (rc) {
        e0->err_ = "tensor-core contraction: output width outside the supported range";
        return rc;
      }
    }
    g.launched = true;
    return 0;
  }
  for (auto& z : g.zero) cudaMemsetAsync(z.first, 0, z.second * sizeof(double), s);
  for (int i = 0; i < 3; ++i) {
    const int rc = e0->launch_kplan(g.st[i], g.fp32, true);
    if (rc) return rc;
  }
  return 0;
}

// y_out_ = H_eff x_in_ for every member of the current grouped plan of `node`
// (which covers the active problems).
int BatchRunner::product(int node, const std::vector<int>& active) {
  auto it = cur_.find(node);
  Grouped* g = it != cur_.end() ? it->second.get() : nullptr;
  bool covered = g != nullptr;
  for (size_t i = 0; covered && i < active.size(); ++i)
    covered = std::find(g->members.begin(), g->members.end(), active[i]) != g->members.end();
  if (g && (!covered || stale(*g) || (double)active.size() < kRebuildFraction * (double)g->members.size())) {
    cudaStreamSynchronize(es_[0]->stream_);
    cur_.erase(it);
    g = nullptr;
  }
  if (!g) {
    std::unique_ptr<Grouped> ng;
    const int rc = build(node, active, &ng);
    if (rc) return rc;
    g = ng.get();
    cur_[node] = std::move(ng);
  }
  Engine* e0 = es_[g->members[0]];
  cudaStream_t s = e0->stream_;
  if (g->exec && g->scratch != e0->scratch_) {
    cudaGraphExecDestroy(g->exec);
    g->exec = nullptr;
  }
  if (g->exec) {
    count_launches((int)g->graph_kernels);
    return e0->check(cudaGraphLaunch(g->exec, s), "batched product graph") ? 0 : -3;
  }
  bool tuned = true;
  for (const KPlan& p : g->st)
    if (!p.outs.empty() && p.shape[g->fp32] < 0 && e0->forced_shape_ < 0) tuned = false;
  if (g->tg && !g->launched) tuned = false;   // first launch eager (one-time kernel set-up on the host)
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  const bool capturable = use_graphs_ && tuned && s != nullptr &&
                          cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone;
  if (!capturable) return launch(*g);
  // every allocation a launch may need happens before the capture
  for (KPlan& p : g->st)
    if (!p.outs.empty()) {
      const int shape = e0->forced_shape_ >= 0 ? e0->forced_shape_ : p.shape[g->fp32];
      e0->ensure_scratch(std::max<long long>(p.variant(shape, s).scratch_need, 1));
    }
  const long long before = launch_count();
  if (!e0->check(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed), "graph capture")) return -3;
  const int rc = launch(*g);
  cudaGraph_t graph = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(s, &graph);
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (!e0->check(ce, "graph capture")) return -3;
  const cudaError_t ie = cudaGraphInstantiate(&g->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (!e0->check(ie, "graph instantiate")) return -3;
  g->graph_kernels = launch_count() - before;   // recorded, not run: counted per replay
  count_launches(-(int)g->graph_kernels);
  g->scratch = e0->scratch_;
  count_launches((int)g->graph_kernels);
  return e0->check(cudaGraphLaunch(g->exec, s), "batched product graph") ? 0 : -3;
}

// Lockstep Lanczos over all problems at `node` (each from its own tensor).
int BatchRunner::lanczos(int node, const std::vector<double>& tol, int max_krylov, bool mixed, int max_restarts,
                         std::vector<double>* energy, std::vector<double>* resid, std::vector<int>* iters) {
  const int B = (int)es_.size();
  struct St {
    long long n = 0;
    int kmax = 0, j = 0, k = 0, restart = 0, stalls = 0, iters = 0;
    double theta = 0.0, res = 0.0, prev_res = 1e300;
    bool active = true;
  };
  std::vector<St> st(B);
  for (int b = 0; b < B; ++b) {
    Engine* e = es_[b];
    e->use_mixed_ = mixed;
    St& z = st[b];
    z.n = e->layout_[node].size;
    z.kmax = std::min(std::max(max_krylov, 2), kMaxKrylov);
    if (z.kmax > z.n) z.kmax = (int)z.n;
    const int rc = e->lz_prepare(z.kmax);
    if (rc) return rc;
    e->lz_start(node);
  }
  cudaStream_t s = es_[0]->stream_;
  for (;;) {
    std::vector<int> active;
    for (int b = 0; b < B; ++b)
      if (st[b].active) active.push_back(b);
    if (active.empty()) break;
    for (int b : active) {
      Engine* e = es_[b];
      launch_copy(e->V_ + (long long)st[b].j * e->nmax_, e->x_in_, st[b].n, s);
    }
    int rc = product(node, active);
    if (rc) return rc;
    for (int b : active) {
      Engine* e = es_[b];
      e->lz_iteration(st[b].j, st[b].n);
      e->lz_queue_check(st[b].j);
      e->lz_next_vector(st[b].j, st[b].n);
      st[b].iters += 1;
    }
    for (int b : active)
      if (!es_[b]->check(cudaEventSynchronize(es_[b]->ev_conv_[st[b].j]), "batched lanczos")) return -3;
    for (int b : active) {
      Engine* e = es_[b];
      St& z = st[b];
      z.k = z.j + 1;
      bool finish = e->lz_converged(z.j, tol[b], &z.theta, &z.res);
      if (!finish && z.j + 1 >= z.kmax) {
        bool stop = z.restart + 1 >= max_restarts;
        if (mixed) {
          const bool near_floor = z.res <= 1e3 * e->mixed_tol * std::fabs(z.theta);
          z.stalls = (near_floor && z.res > 0.98 * z.prev_res) ? z.stalls + 1 : 0;
          if (z.stalls >= 2) stop = true;
        }
        z.prev_res = std::min(z.prev_res, z.res);
        if (!stop) {
          int j0 = 0;
          if ((rc = e->lz_thick_restart(z.k, z.kmax, z.n, &j0))) return rc;
          z.j = j0;
          z.restart += 1;
          continue;
        }
        finish = true;
      }
      if (finish) {
        e->lz_finish(node, z.k);
        z.active = false;
      } else {
        z.j += 1;
      }
    }
  }
  if (!es_[0]->check(cudaStreamSynchronize(s), "batched lanczos end")) return -3;
  energy->assign(B, 0.0);
  resid->assign(B, 0.0);
  iters->assign(B, 0);
  for (int b = 0; b < B; ++b) {
    Engine* e = es_[b];
    e->use_mixed_ = false;
    e->last_conv_ = -1;
    (*energy)[b] = e->ring_host_[4 * kMaxKrylov];
    (*resid)[b] = e->ring_host_[4 * kMaxKrylov + 1];
    (*iters)[b] = st[b].iters;
  }
  return 0;
}

int BatchRunner::optimize(int node, double tol, int max_krylov, std::vector<SweepStats>* stats) {
  const int B = (int)es_.size();
  for (Engine* e : es_) {
    const int rc = e->move_to(node);
    if (rc) return rc;
  }
  const bool mixed = es_[0]->precision_ != PREC_FP64;
  std::vector<double> energy, res, tols(B, tol);
  std::vector<int> iters, mixed_iters(B, 0);
  int rc = 0;
  if (mixed) {
    for (int b = 0; b < B; ++b) tols[b] = std::max(0.3 * tol, es_[b]->mixed_tol);
    cudaMemsetAsync(es_[0]->d_err_, 0, sizeof(int), es_[0]->stream_);
    if ((rc = lanczos(node, tols, max_krylov, true, 50, &energy, &res, &mixed_iters))) return rc;
    int herr = 0;
    cudaMemcpyAsync(&herr, es_[0]->d_err_, sizeof(int), cudaMemcpyDeviceToHost, es_[0]->stream_);
    if (!es_[0]->check(cudaStreamSynchronize(es_[0]->stream_), "batched mixed phase")) return -3;
    if (herr) {
      es_[0]->err_ = "tensor-core H_eff: an mbarrier wait hit its iteration limit";
      return -6;
    }
    iters.assign(B, 0);
    for (int b = 0; b < B; ++b) {
      double e = 0.0, r = 0.0;
      int it = 0;
      // the residual correction with float-float products, as in an unbatched update
      es_[b]->ff_products_ = true;
      rc = es_[b]->lanczos(node, tol, max_krylov, false, 50, &e, &r, &it);
      es_[b]->ff_products_ = false;
      if (rc) return rc;
      energy[b] = e;
      res[b] = r;
      iters[b] = it;
    }
  } else {
    for (int b = 0; b < B; ++b) tols[b] = tol;
    if ((rc = lanczos(node, tols, max_krylov, false, 50, &energy, &res, &iters))) return rc;
  }
  for (int b = 0; b < B; ++b) {
    Engine* e = es_[b];
    e->last_lanczos_iters = iters[b];
    e->last_mixed_iters = mixed_iters[b];
    e->last_residual = res[b] / std::max(1e-300, std::fabs(energy[b]));
    SweepStats& z = (*stats)[b];
    z.matvecs += iters[b] + mixed_iters[b];
    z.matvecs_mixed += mixed_iters[b];
    z.node_updates += 1;
    z.energy = energy[b];
    z.max_residual = std::max(z.max_residual, e->last_residual);
    if (res[b] > tol * std::fabs(energy[b])) z.not_converged += 1;
  }
  return 0;
}

int BatchRunner::sweep(double tol, int max_krylov, std::vector<SweepStats>* stats) {
  if (es_.empty()) return 0;
  for (int node : sweep_order(es_[0]->nodes_)) {
    const int rc = optimize(node, tol, max_krylov, stats);
    if (rc) return rc;
  }
  return 0;
}

}  // namespace qed
