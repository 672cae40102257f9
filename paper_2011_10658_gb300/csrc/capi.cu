// C ABI of the qedttn library (see include/qedttn.h for the contract).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <exception>
#include <string>
#include <vector>

#include "../../include/qedttn.h"
#include "batch.h"
#include "engine.h"
#include "model.h"
#include "state.h"

namespace {
thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

int engine_status(qed::Engine* e, int rc) {
  if (rc == 0) return QED_OK;
  g_err = e->error();
  if (rc == -2) return QED_ENOMEM;
  if (rc == -5) return QED_ENAN;
  if (rc == -7) return QED_EUNSUPPORTED;
  if (rc == -6) return QED_ETIMEOUT;
  if (rc == -1) return QED_EINVAL;
  return QED_ECUDA;
}

bool pow2(int v) { return v >= 1 && (v & (v - 1)) == 0; }
}  // namespace

void qed_set_last_error(const char* msg) { g_err = msg; }


#define QED_TRY(...)                                    \
  try {                                                 \
    __VA_ARGS__                                         \
  } catch (const std::bad_alloc&) {                     \
    return fail(QED_ENOMEM, "out of host memory");      \
  } catch (const qed::DeviceAllocError& ex) {           \
    return fail(QED_ENOMEM, ex.what());                 \
  } catch (const std::exception& ex) {                  \
    return fail(QED_EINVAL, ex.what());                 \
  } catch (...) {                                       \
    return fail(QED_EINVAL, "unknown error");           \
  }

extern "C" {

#define QED_API __attribute__((visibility("default")))

QED_API const char* qed_last_error(void) { return g_err.c_str(); }

QED_API int qed_basis(int parity, int8_t* table, int32_t* n_rows) {
  if (parity != 1 && parity != -1) return fail(QED_EINVAL, "parity must be +1 or -1");
  if (n_rows) *n_rows = qed::kLocalDim;
  if (!table) return QED_OK;
  QED_TRY(qed::enumerate_basis(parity, table); return QED_OK;)
}

QED_API int qed_local_op(int parity, int op_kind, int j1, int j2, int16_t* src, double* val) {
  if (parity != 1 && parity != -1) return fail(QED_EINVAL, "parity must be +1 or -1");
  if (!src || !val) return fail(QED_EINVAL, "null output");
  if (op_kind < QED_OP_IDENTITY || (op_kind > QED_OP_E2 && op_kind != QED_OP_PC))
    return fail(QED_EINVAL, "unknown op kind");
  if (op_kind != QED_OP_E2 && (j1 < 0 || j1 > 5)) return fail(QED_EINVAL, "half-link index out of range");
  if (op_kind == QED_OP_C && (j2 < 0 || j2 > 5 || j1 == j2)) return fail(QED_EINVAL, "C needs two distinct half-links");
  if ((op_kind == QED_OP_P || op_kind == QED_OP_PC) && (j2 < 0 || j2 > 2)) return fail(QED_EINVAL, "P needs k in 0..2");
  if (op_kind == QED_OP_E2 && (j1 < 0 || j1 > 63)) return fail(QED_EINVAL, "E2 mask out of range");
  QED_TRY(
    qed::OpKey k;
    k.kind = op_kind;
    k.a = j1;
    k.b = j2;
    qed::SiteOp op;
    qed::build_site_op(parity, k, &op);
    for (int i = 0; i < qed::kLocalDim; ++i) {
      src[i] = op.src[i];
      val[i] = op.val[i];
    }
    return QED_OK;)
}

QED_API int qed_model_create(const qed_params* p, qed_model** out) {
  if (!p || !out) return fail(QED_EINVAL, "null argument");
  *out = nullptr;
  if (p->boundary != 0 && p->boundary != 1) return fail(QED_EINVAL, "boundary must be 0 (open) or 1 (periodic)");
  if (!pow2(p->Lx) || !pow2(p->Ly) || !pow2(p->Lz) || p->Lx * p->Ly * p->Lz < 2 || p->Lx * p->Ly * p->Lz > 4096)
    return fail(QED_EINVAL, "lattice extents must be powers of two, 2 <= sites <= 4096");
  const double c[5] = {p->t, p->m, p->ge2, p->cB, p->nu};
  for (double v : c)
    if (!std::isfinite(v)) return fail(QED_ENAN, "non-finite coupling");
  QED_TRY(
    qed_model* m = new qed_model;
    m->p.Lx = p->Lx; m->p.Ly = p->Ly; m->p.Lz = p->Lz; m->p.boundary = p->boundary;
    m->p.t = p->t; m->p.m = p->m; m->p.ge2 = p->ge2; m->p.cB = p->cB; m->p.nu = p->nu; m->p.Q = p->Q;
    qed::build_terms(m->p, &m->terms, &m->constant);
    m->nodes = qed::build_tree(p->Lx, p->Ly, p->Lz);
    *out = m;
    return QED_OK;)
}

QED_API void qed_model_destroy(qed_model* m) { delete m; }

QED_API int qed_model_set_site_potential(qed_model* m, const double* mu, int32_t n) {
  if (!m) return fail(QED_EINVAL, "null model");
  const int N = m->p.Lx * m->p.Ly * m->p.Lz;
  if (n != 0 && (n != N || !mu)) return fail(QED_EINVAL, "need one chemical potential per site (or n = 0)");
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(mu[i])) return fail(QED_ENAN, "non-finite chemical potential");
  QED_TRY(
    m->p.mu.assign(mu, mu + n);
    qed::build_terms(m->p, &m->terms, &m->constant);
    return QED_OK;)
}

QED_API int qed_model_info(const qed_model* m, int32_t* n_sites, int32_t* n_terms, int32_t* n_nodes, double* constant) {
  if (!m) return fail(QED_EINVAL, "null model");
  if (n_sites) *n_sites = m->p.Lx * m->p.Ly * m->p.Lz;
  if (n_terms) *n_terms = (int32_t)m->terms.size();
  if (n_nodes) *n_nodes = (int32_t)m->nodes.size();
  if (constant) *constant = m->constant;
  return QED_OK;
}

QED_API int qed_model_terms(const qed_model* m, double* coef, int32_t* cls, int32_t* n_ops, int32_t* ops, int64_t cap,
                    int64_t* n) {
  if (!m) return fail(QED_EINVAL, "null model");
  if (n) *n = (int64_t)m->terms.size();
  if (!coef || cap <= 0) return QED_OK;
  if (cap < (int64_t)m->terms.size()) return fail(QED_EINVAL, "buffer too small");
  for (size_t i = 0; i < m->terms.size(); ++i) {
    const qed::Term& t = m->terms[i];
    coef[i] = t.coef;
    if (cls) cls[i] = t.cls;
    if (n_ops) n_ops[i] = (int32_t)t.ops.size();
    if (ops)
      for (size_t f = 0; f < 4; ++f) {
        int32_t* o = ops + (i * 4 + f) * 4;
        if (f < t.ops.size()) {
          o[0] = t.ops[f].first; o[1] = t.ops[f].second.kind; o[2] = t.ops[f].second.a; o[3] = t.ops[f].second.b;
        } else {
          o[0] = o[1] = o[2] = o[3] = -1;
        }
      }
  }
  return QED_OK;
}

QED_API int qed_model_tree(const qed_model* m, int32_t* nodes, int64_t cap, int64_t* n) {
  if (!m) return fail(QED_EINVAL, "null model");
  if (n) *n = (int64_t)m->nodes.size();
  if (!nodes || cap <= 0) return QED_OK;
  if (cap < (int64_t)m->nodes.size()) return fail(QED_EINVAL, "buffer too small");
  for (size_t i = 0; i < m->nodes.size(); ++i) {
    const qed::TreeNode& t = m->nodes[i];
    int32_t* o = nodes + 7 * i;
    o[0] = t.layer; o[1] = t.axis; o[2] = t.child_kind[0]; o[3] = t.child[0];
    o[4] = t.child_kind[1]; o[5] = t.child[1]; o[6] = t.parent;
  }
  return QED_OK;
}

QED_API int qed_model_sweep_order(const qed_model* m, int32_t* order, int64_t cap, int64_t* n) {
  if (!m) return fail(QED_EINVAL, "null model");
  const std::vector<int> o = qed::sweep_order(m->nodes);
  if (n) *n = (int64_t)o.size();
  if (!order || cap <= 0) return QED_OK;
  if (cap < (int64_t)o.size()) return fail(QED_EINVAL, "buffer too small");
  for (size_t i = 0; i < o.size(); ++i) order[i] = o[i];
  return QED_OK;
}

QED_API int qed_model_sectors(const qed_model* m, int32_t chi, int32_t* triples, int64_t cap, int64_t* n) {
  if (!m) return fail(QED_EINVAL, "null model");
  if (chi < 1 || chi > 4096) return fail(QED_EINVAL, "chi out of range");
  QED_TRY(
    std::vector<qed::Sectors> bonds;
    std::string err;
    if (!qed::sector_table(m->p, chi, m->nodes, &bonds, &err)) return fail(QED_EUNSUPPORTED, err);
    int64_t total = 0;
    for (auto& b : bonds) total += (int64_t)b.q.size();
    if (n) *n = total;
    if (!triples || cap <= 0) return QED_OK;
    if (cap < total) return fail(QED_EINVAL, "buffer too small");
    int64_t k = 0;
    for (size_t i = 0; i < bonds.size(); ++i)
      for (size_t j = 0; j < bonds[i].q.size(); ++j) {
        triples[3 * k] = (int32_t)i;
        triples[3 * k + 1] = bonds[i].q[j];
        triples[3 * k + 2] = bonds[i].dim[j];
        ++k;
      }
    return QED_OK;)
}

QED_API int ttn_create(const qed_model* m, int32_t chi, uint64_t seed, int precision, void* cuda_stream, ttn_state** out) {
  if (!m || !out) return fail(QED_EINVAL, "null argument");
  *out = nullptr;
  if (chi < 1 || chi > 512) return fail(QED_EINVAL, "chi out of range (1..512)");
  if (precision != QED_PREC_FP64 && precision != QED_PREC_TF32 && precision != QED_PREC_BF16 &&
      precision != QED_PREC_TF32X3)
    return fail(QED_EINVAL, "unknown precision");
  int dev_count = 0;
  if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count == 0)
    return fail(QED_ECUDA, "no CUDA device available");
  QED_TRY(
    ttn_state* s = new ttn_state;
    try {
      s->engine = new qed::Engine(m->p, chi, seed, precision, (cudaStream_t)cuda_stream);
    } catch (...) {
      delete s;
      throw;
    }
    s->model = m;
    *out = s;
    return QED_OK;)
}

QED_API void ttn_destroy(ttn_state* s) {
  if (!s) return;
  delete s->engine;
  delete s;
}

QED_API int ttn_sweep(ttn_state* s, int32_t n_sweeps, double tol, int32_t max_krylov, ttn_sweep_stats* out) {
  if (!s) return fail(QED_EINVAL, "null state");
  if (n_sweeps < 0 || !(tol > 0.0) || max_krylov < 2 || max_krylov > 128)
    return fail(QED_EINVAL, "n_sweeps >= 0, tol > 0, 2 <= max_krylov <= 128");
  QED_TRY(
    auto t0 = std::chrono::steady_clock::now();
    qed::SweepStats st;
    for (int i = 0; i < n_sweeps; ++i) {
      int rc = s->engine->sweep(tol, max_krylov, &st, nullptr);
      if (rc) return engine_status(s->engine, rc);
    }
    auto t1 = std::chrono::steady_clock::now();
    if (out) {
      out->energy = st.energy;
      out->matvecs = st.matvecs;
      out->matvecs_mixed = st.matvecs_mixed;
      out->node_updates = st.node_updates;
      out->not_converged = st.not_converged;
      out->max_rel_residual = st.max_residual;
      out->seconds = std::chrono::duration<double>(t1 - t0).count();
    }
    if (st.not_converged) return fail(QED_ENOCONV, "some node updates stopped above tolerance");
    return QED_OK;)
}

QED_API int ttn_set_precision(ttn_state* s, int precision) {
  if (!s) return fail(QED_EINVAL, "null state");
  if (precision != QED_PREC_FP64 && precision != QED_PREC_TF32 && precision != QED_PREC_BF16 &&
      precision != QED_PREC_TF32X3)
    return fail(QED_EINVAL, "unknown precision");
  s->engine->set_precision(precision);
  return QED_OK;
}

QED_API int ttn_set_mixed_tol(ttn_state* s, double mixed_tol) {
  if (!s) return fail(QED_EINVAL, "null state");
  if (!(mixed_tol > 0.0) || !(mixed_tol < 1.0)) return fail(QED_EINVAL, "mixed_tol must lie in (0, 1)");
  s->engine->mixed_tol = mixed_tol;
  return QED_OK;
}

QED_API int ttn_set_couplings(ttn_state* s, const double couplings[5]) {
  if (!s || !couplings) return fail(QED_EINVAL, "null argument");
  QED_TRY(
    qed::Engine* e = s->engine;
    int rc = e->move_to(e->n_nodes() - 1);   // operators are rebuilt towards the root
    if (rc) return engine_status(e, rc);
    qed::Params np = e->params();
    np.t = couplings[0]; np.m = couplings[1]; np.ge2 = couplings[2]; np.cB = couplings[3]; np.nu = couplings[4];
    rc = e->set_couplings(np);
    if (rc == -1) return fail(QED_EINVAL, e->error().c_str());
    return engine_status(e, rc);)
}

namespace {

int drive_check(const qed_drive* d) {
  if (!d) return fail(QED_EINVAL, "null drive settings");
  if (!(d->nu_start > 0.0) || !(d->nu_step > 0.0) || !(d->quad_coef > 0.0) || !(d->nu_max >= d->nu_start) ||
      !std::isfinite(d->nu_max))
    return fail(QED_EINVAL, "need 0 < nu_start <= nu_max (finite), nu_step > 0, quad_coef > 0");
  if (!(d->tol_start > 0.0) || !(d->tol_final > 0.0) || !(d->tol_factor > 0.0) || !(d->tol_factor <= 1.0))
    return fail(QED_EINVAL, "need tol_start > 0, tol_final > 0, 0 < tol_factor <= 1");
  if (!(d->conv_rel >= 0.0) || !(d->rise_rel >= 0.0) || d->min_final_sweeps < 2 || d->max_sweeps < 1)
    return fail(QED_EINVAL, "need conv_rel >= 0, rise_rel >= 0, min_final_sweeps >= 2, max_sweeps >= 1");
  return QED_OK;
}

double drive_tol(const qed_drive* d, int sweep) {
  return std::max(d->tol_final, d->tol_start * std::pow(d->tol_factor, (double)sweep));
}

}  // namespace

QED_API int qed_drive_start(const qed_drive* d, qed_drive_state* st) {
  if (int rc = drive_check(d)) return rc;
  if (!st) return fail(QED_EINVAL, "null state");
  std::memset(st, 0, sizeof(*st));
  st->nu = d->nu_start;
  if (st->nu >= d->nu_max) {
    st->nu = d->nu_max;
    st->stage = 2;
  }
  st->tol = drive_tol(d, 0);
  return QED_OK;
}

QED_API int qed_drive_next(const qed_drive* d, qed_drive_state* st, double energy) {
  if (int rc = drive_check(d)) return rc;
  if (!st || !std::isfinite(energy)) return fail(QED_EINVAL, "null state or non-finite energy");
  if (st->done) return QED_OK;
  if (st->stage == 2) {
    // the sweep just run was at nu_max
    st->final_sweeps += 1;
    if (st->final_sweeps >= d->min_final_sweeps && std::fabs(energy - st->e_prev) <= d->conv_rel * std::fabs(energy))
      st->done = 1;
  } else {
    double next;
    if (st->stage == 0 && st->sweep > 0 && energy - st->e_prev > d->rise_rel * std::fabs(st->e_prev)) {
      // the energy rose: quadratic growth from the nu of this sweep
      st->stage = 1;
      st->nu_switch = st->nu;
      st->since_switch = 1;
      next = st->nu_switch + d->quad_coef * d->nu_step;
    } else if (st->stage == 0) {
      next = st->nu + d->nu_step;
    } else {
      st->since_switch += 1;
      const double k = (double)st->since_switch;
      next = st->nu_switch + d->quad_coef * d->nu_step * k * k;
    }
    if (next >= d->nu_max) {
      next = d->nu_max;
      st->stage = 2;
    }
    st->nu = next;
  }
  st->e_prev = energy;
  st->sweep += 1;
  st->tol = drive_tol(d, st->sweep);
  return QED_OK;
}

QED_API int ttn_drive(ttn_state* s, const qed_drive* d, qed_drive_record* log, int32_t cap, int32_t* n) {
  if (!s || !n || (cap > 0 && !log) || cap < 0) return fail(QED_EINVAL, "null argument or negative cap");
  if (int rc = drive_check(d)) return rc;
  if (d->max_krylov < 2 || d->max_krylov > 128) return fail(QED_EINVAL, "2 <= max_krylov <= 128");
  *n = 0;
  qed_drive_state st;
  qed_drive_start(d, &st);
  while (!st.done && st.sweep < d->max_sweeps) {
    const qed::Params& p = s->engine->params();
    if (p.nu != st.nu) {
      const double c[5] = {p.t, p.m, p.ge2, p.cB, st.nu};
      if (int rc = ttn_set_couplings(s, c)) return rc;
    }
    ttn_sweep_stats ss;
    int rc = ttn_sweep(s, 1, st.tol, d->max_krylov, &ss);
    if (rc != QED_OK && rc != QED_ENOCONV) return rc;
    double et = 0.0, ew = 0.0;
    if ((rc = ttn_energy(s, &et, &ew, nullptr))) return rc;
    double sc[4];
    int64_t ns = 0;
    if ((rc = ttn_measure(s, QED_MEAS_SCALARS, sc, 4, &ns))) return rc;
    if (*n < cap) {
      qed_drive_record& r = log[*n];
      r.sweep = st.sweep;
      r.stage = st.stage;
      r.nu = st.nu;
      r.tol = st.tol;
      r.energy = et;
      r.energy_without_penalty = ew;
      r.delta_L = sc[1];
      r.matvecs = ss.matvecs;
      r.not_converged = ss.not_converged;
      r.max_rel_residual = ss.max_rel_residual;
      r.seconds = ss.seconds;
    }
    *n += 1;
    qed_drive_next(d, &st, et);
  }
  if (!st.done) return fail(QED_ENOCONV, "driven optimisation: max_sweeps reached before convergence");
  return QED_OK;
}

QED_API int ttn_set_wait_limit(ttn_state* s, int64_t polls) {
  if (!s) return fail(QED_EINVAL, "null state");
  s->engine->wait_polls = polls < 0 ? -1 : polls;
  return QED_OK;
}

QED_API int ttn_last_update(ttn_state* s, int32_t* iters_fp64, int32_t* iters_mixed, double* rel_residual,
                            double* ritz_mixed, double* rel_residual_mixed) {
  if (!s) return fail(QED_EINVAL, "null state");
  if (iters_fp64) *iters_fp64 = s->engine->last_lanczos_iters;
  if (iters_mixed) *iters_mixed = s->engine->last_mixed_iters;
  if (rel_residual) *rel_residual = s->engine->last_residual;
  if (ritz_mixed) *ritz_mixed = s->engine->last_mixed_ritz;
  if (rel_residual_mixed) *rel_residual_mixed = s->engine->last_mixed_residual;
  return QED_OK;
}

QED_API int ttn_set_profiling(ttn_state* s, int on) {
  if (!s) return fail(QED_EINVAL, "null state");
  s->engine->set_profiling(on != 0);
  return QED_OK;
}

QED_API int ttn_reset_timing(ttn_state* s) {
  if (!s) return fail(QED_EINVAL, "null state");
  QED_TRY(s->engine->reset_timing(); return QED_OK;)
}

QED_API int ttn_kernel_timing(ttn_state* s, int kernel_class, double* ms, int64_t* launches, double* flops_alg,
                              double* flops_exec, double* bytes_alg) {
  if (!s) return fail(QED_EINVAL, "null state");
  if (kernel_class < 0 || kernel_class >= qed::KC_COUNT) return fail(QED_EINVAL, "unknown kernel class");
  QED_TRY(
    qed::KernelTiming t[qed::KC_COUNT];
    int rc = s->engine->kernel_timing(t);
    if (rc) return engine_status(s->engine, rc);
    const qed::KernelTiming& k = t[kernel_class];
    if (ms) *ms = k.ms;
    if (launches) *launches = k.launches;
    if (flops_alg) *flops_alg = k.flops_alg;
    if (flops_exec) *flops_exec = k.flops_exec;
    if (bytes_alg) *bytes_alg = k.bytes_alg;
    return QED_OK;)
}

QED_API int ttn_batch_sweep(ttn_state* const* states, int32_t n, int32_t n_sweeps, double tol, int32_t max_krylov,
                            ttn_sweep_stats* out) {
  if (!states || n < 1) return fail(QED_EINVAL, "need at least one state");
  if (n_sweeps < 0 || !(tol > 0.0) || max_krylov < 2 || max_krylov > 128)
    return fail(QED_EINVAL, "n_sweeps >= 0, tol > 0, 2 <= max_krylov <= 128");
  std::vector<qed::Engine*> es;
  for (int i = 0; i < n; ++i) {
    if (!states[i]) return fail(QED_EINVAL, "null state");
    const qed::Params& a = states[0]->model->p;
    const qed::Params& b = states[i]->model->p;
    if (a.Lx != b.Lx || a.Ly != b.Ly || a.Lz != b.Lz) return fail(QED_EINVAL, "states differ in lattice size");
    if (states[i]->engine->precision() != states[0]->engine->precision())
      return fail(QED_EINVAL, "states differ in precision");
    if (states[i]->engine->stream() != states[0]->engine->stream()) return fail(QED_EINVAL, "states differ in stream");
    for (int j = 0; j < i; ++j)
      if (states[j] == states[i]) return fail(QED_EINVAL, "a state appears twice");
    es.push_back(states[i]->engine);
  }
  QED_TRY(
    auto t0 = std::chrono::steady_clock::now();
    std::vector<qed::SweepStats> st(n);
    qed::BatchRunner runner(es);
    for (int i = 0; i < n_sweeps; ++i) {
      int rc = runner.sweep(tol, max_krylov, &st);
      if (rc) {
        for (qed::Engine* e : es)
          if (!e->error().empty()) return engine_status(e, rc);
        return engine_status(es[0], rc);
      }
    }
    auto t1 = std::chrono::steady_clock::now();
    int bad = 0;
    for (int i = 0; i < n; ++i) {
      if (out) {
        out[i].energy = st[i].energy;
        out[i].matvecs = st[i].matvecs;
        out[i].matvecs_mixed = st[i].matvecs_mixed;
        out[i].node_updates = st[i].node_updates;
        out[i].not_converged = st[i].not_converged;
        out[i].max_rel_residual = st[i].max_residual;
        out[i].seconds = std::chrono::duration<double>(t1 - t0).count();
      }
      bad += st[i].not_converged;
    }
    if (bad) return fail(QED_ENOCONV, "some node updates stopped above tolerance");
    return QED_OK;)
}

QED_API int ttn_optimize_node(ttn_state* s, int32_t node, double tol, int32_t max_krylov, double* energy) {
  if (!s) return fail(QED_EINVAL, "null state");
  if (node < 0 || node >= s->engine->n_nodes()) return fail(QED_EINVAL, "node out of range");
  if (!(tol > 0.0) || max_krylov < 2 || max_krylov > 128) return fail(QED_EINVAL, "bad tolerance or Krylov size");
  QED_TRY(
    qed::SweepStats st;
    double e = 0;
    int rc = s->engine->optimize_node(node, tol, max_krylov, &st, &e);
    if (rc) return engine_status(s->engine, rc);
    if (energy) *energy = e;
    if (st.not_converged) return fail(QED_ENOCONV, "node update stopped above tolerance");
    return QED_OK;)
}

QED_API int ttn_move_center(ttn_state* s, int32_t node) {
  if (!s) return fail(QED_EINVAL, "null state");
  if (node < 0 || node >= s->engine->n_nodes()) return fail(QED_EINVAL, "node out of range");
  QED_TRY(return engine_status(s->engine, s->engine->move_to(node));)
}

QED_API int ttn_info(ttn_state* s, int32_t* center, int32_t* n_nodes, int64_t* max_node_size) {
  if (!s) return fail(QED_EINVAL, "null state");
  if (center) *center = s->engine->center();
  if (n_nodes) *n_nodes = s->engine->n_nodes();
  if (max_node_size) {
    int64_t mx = 0;
    for (int i = 0; i < s->engine->n_nodes(); ++i) mx = std::max<int64_t>(mx, s->engine->node_size(i));
    *max_node_size = mx;
  }
  return QED_OK;
}

QED_API int ttn_node_size(ttn_state* s, int32_t node, int64_t* n) {
  if (!s || !n) return fail(QED_EINVAL, "null argument");
  if (node < 0 || node >= s->engine->n_nodes()) return fail(QED_EINVAL, "node out of range");
  *n = s->engine->node_size(node);
  return QED_OK;
}

QED_API int ttn_energy(ttn_state* s, double* E_total, double* E_without_penalty, double* E_class) {
  if (!s) return fail(QED_EINVAL, "null state");
  QED_TRY(
    double tot = 0, parts[qed::N_CLASSES];
    int rc = s->engine->energy(&tot, parts);
    if (rc) return engine_status(s->engine, rc);
    if (E_total) *E_total = tot;
    if (E_without_penalty) *E_without_penalty = tot - parts[qed::CLS_NU];
    if (E_class)
      for (int c = 0; c < qed::N_COUPLINGS; ++c) E_class[c] = parts[c];
    return QED_OK;)
}

QED_API int ttn_measure(ttn_state* s, int kind, double* out, int64_t cap, int64_t* n) {
  if (!s) return fail(QED_EINVAL, "null state");
  const qed::Params& p = s->model->p;
  qed::Lattice lat{p.Lx, p.Ly, p.Lz, p.boundary == 1};
  const int N = lat.n_sites();
  int64_t need = 0;
  int layers = 0;
  {
    const int mn = std::min(p.Lx, std::min(p.Ly, p.Lz));
    layers = (mn + 1) / 2;
  }
  switch (kind) {
    case QED_MEAS_PROBS: need = (int64_t)N * qed::kLocalDim; break;
    case QED_MEAS_PHI: case QED_MEAS_NX: case QED_MEAS_QX: need = N; break;
    case QED_MEAS_K: need = (int64_t)N * 6; break;
    case QED_MEAS_ELINK: need = lat.n_links(); break;
    case QED_MEAS_SCALARS: need = 4; break;
    case QED_MEAS_SIGMA: need = layers; break;
    default: return fail(QED_EINVAL, "unknown measurement kind");
  }
  if (n) *n = need;
  if (!out || cap <= 0) return QED_OK;
  if (cap < need) return fail(QED_EINVAL, "buffer too small");
  QED_TRY(
    std::vector<double> probs;
    int rc = s->engine->site_probabilities(&probs);
    if (rc) return engine_status(s->engine, rc);
    if (kind == QED_MEAS_PROBS) {
      std::memcpy(out, probs.data(), need * sizeof(double));
      return QED_OK;
    }
    std::vector<int8_t> tab[2];
    for (int t = 0; t < 2; ++t) {
      tab[t].resize(qed::kLocalDim * 9);
      qed::enumerate_basis(t == 0 ? 1 : -1, tab[t].data());
    }
    std::vector<double> phi(N), q(N), k(N * 6);
    for (int x = 0; x < N; ++x) {
      const int8_t* tb = tab[lat.parity(x) == 1 ? 0 : 1].data();
      double a = 0, b = 0, kk[6] = {0, 0, 0, 0, 0, 0};
      for (int r = 0; r < qed::kLocalDim; ++r) {
        const double pr = probs[(size_t)x * qed::kLocalDim + r];
        a += pr * tb[9 * r];
        b += pr * tb[9 * r + 8];
        for (int j = 0; j < 6; ++j) kk[j] += pr * tb[9 * r + 1 + j];
      }
      phi[x] = a;
      q[x] = b;
      for (int j = 0; j < 6; ++j) k[x * 6 + j] = kk[j];
    }
    if (kind == QED_MEAS_PHI) { for (int x = 0; x < N; ++x) out[x] = phi[x]; return QED_OK; }
    if (kind == QED_MEAS_QX) { for (int x = 0; x < N; ++x) out[x] = q[x]; return QED_OK; }
    if (kind == QED_MEAS_NX) {
      for (int x = 0; x < N; ++x) { int par = lat.parity(x); out[x] = 0.5 * (1 + par) - par * phi[x]; }
      return QED_OK;
    }
    if (kind == QED_MEAS_K) { for (int i = 0; i < N * 6; ++i) out[i] = k[i]; return QED_OK; }
    double dL = 0.0;
    int li = 0;
    std::vector<double> elink;
    for (int x = 0; x < N; ++x)
      for (int mu = 0; mu < 3; ++mu) {
        int y = lat.neighbour(x, mu, +1);
        if (y < 0) continue;
        const double kx = k[x * 6 + 3 + mu], ky = k[y * 6 + mu];
        elink.push_back(1.0 - kx);
        dL += std::fabs(kx + ky - 2.0);
        ++li;
      }
    if (kind == QED_MEAS_ELINK) { for (size_t i = 0; i < elink.size(); ++i) out[i] = elink[i]; return QED_OK; }
    if (kind == QED_MEAS_SCALARS) {
      double rho = 0, qs = 0;
      for (int x = 0; x < N; ++x) {
        int par = lat.parity(x);
        rho += 0.5 * (1 + par) - par * phi[x];
        qs += q[x];
      }
      out[0] = rho / N;
      out[1] = dL;
      out[2] = qs;
      out[3] = layers;
      return QED_OK;
    }
    // sigma(l): mean <psi^dag psi> over sites at distance l from the closest boundary
    std::vector<double> sum(layers, 0.0), cnt(layers, 0.0);
    for (int x = 0; x < N; ++x) {
      int c[3];
      lat.coords(x, c);
      const int dims[3] = {p.Lx, p.Ly, p.Lz};
      int l = 1 << 30;
      for (int a = 0; a < 3; ++a) l = std::min(l, std::min(c[a], dims[a] - 1 - c[a]));
      if (l < layers) { sum[l] += phi[x]; cnt[l] += 1; }
    }
    for (int l = 0; l < layers; ++l) out[l] = cnt[l] > 0 ? sum[l] / cnt[l] : 0.0;
    return QED_OK;)
}

QED_API int ttn_node_export(ttn_state* s, int32_t node, double* buf, int64_t cap, int64_t* n) {
  if (!s) return fail(QED_EINVAL, "null state");
  if (node < 0 || node >= s->engine->n_nodes()) return fail(QED_EINVAL, "node out of range");
  const int64_t need = s->engine->node_size(node);
  if (n) *n = need;
  if (!buf || cap <= 0) return QED_OK;
  if (cap < need) return fail(QED_EINVAL, "buffer too small");
  QED_TRY(
    std::vector<double> h;
    int rc = s->engine->node_export(node, &h);
    if (rc) return engine_status(s->engine, rc);
    std::memcpy(buf, h.data(), need * sizeof(double));
    return QED_OK;)
}

QED_API int ttn_node_import(ttn_state* s, int32_t node, const double* buf, int64_t n) {
  if (!s || !buf) return fail(QED_EINVAL, "null argument");
  if (node < 0 || node >= s->engine->n_nodes()) return fail(QED_EINVAL, "node out of range");
  if (n != s->engine->node_size(node)) return fail(QED_EINVAL, "size mismatch");
  QED_TRY(
    std::vector<double> h(buf, buf + n);
    int rc = s->engine->node_import(node, h);
    if (rc == -5) return fail(QED_ENAN, "non-finite tensor entry");
    if (rc == -1) return fail(QED_EINVAL, "size mismatch");
    return engine_status(s->engine, rc);)
}

QED_API int ttn_load_tensors(ttn_state* s, const double* const* bufs, const int64_t* sizes, int32_t n_nodes) {
  if (!s || !bufs || !sizes) return fail(QED_EINVAL, "null argument");
  if (n_nodes != s->engine->n_nodes()) return fail(QED_EINVAL, "n_nodes mismatch");
  QED_TRY(
    std::vector<long long> sz(sizes, sizes + n_nodes);
    int rc = s->engine->load_tensors(bufs, sz.data(), n_nodes);
    if (rc == -1) return fail(QED_EINVAL, "tensor size mismatch");
    if (rc == -5) return fail(QED_ENAN, "non-finite tensor entry");
    return engine_status(s->engine, rc);)
}

QED_API int qed_launch_count(int64_t* count) {
  if (!count) return fail(QED_EINVAL, "null argument");
  *count = qed::launch_count();
  return QED_OK;
}

QED_API int ttn_apply_heff(ttn_state* s, const double* x, double* y, int64_t n) {
  if (!s || !x || !y) return fail(QED_EINVAL, "null argument");
  const int64_t need = s->engine->node_size(s->engine->center());
  if (n != need) return fail(QED_EINVAL, "size must equal the centre tensor size");
  QED_TRY(
    double *dx = nullptr, *dy = nullptr;
    if (cudaMalloc(&dx, n * sizeof(double)) != cudaSuccess) return fail(QED_ENOMEM, "device allocation");
    if (cudaMalloc(&dy, n * sizeof(double)) != cudaSuccess) { cudaFree(dx); return fail(QED_ENOMEM, "device allocation"); }
    cudaStream_t st = s->engine->stream();
    cudaMemcpyAsync(dx, x, n * sizeof(double), cudaMemcpyHostToDevice, st);
    int rc = s->engine->apply_heff_native(dx, dy);
    if (!rc) cudaMemcpyAsync(y, dy, n * sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    cudaFree(dx);
    cudaFree(dy);
    if (rc) return engine_status(s->engine, rc);
    if (e != cudaSuccess) return fail(QED_ECUDA, cudaGetErrorString(e));
    return QED_OK;)
}

QED_API int ttn_apply_heff_device(ttn_state* s, const double* x_device, double* y_device, int64_t n) {
  if (!s || !x_device || !y_device) return fail(QED_EINVAL, "null argument");
  if (n != s->engine->node_size(s->engine->center())) return fail(QED_EINVAL, "size must equal the centre tensor size");
  QED_TRY(return engine_status(s->engine, s->engine->apply_heff_native(x_device, y_device));)
}

namespace {
const char kCkptTag[8] = {'Q', 'E', 'D', 'T', 'T', 'N', '0', '1'};

struct Fnv {
  uint64_t h = 1469598103934665603ull;
  void add(const void* p, size_t n) {
    const unsigned char* b = (const unsigned char*)p;
    for (size_t i = 0; i < n; ++i) { h ^= b[i]; h *= 1099511628211ull; }
  }
};

bool write_all(FILE* f, Fnv* fnv, const void* p, size_t n) {
  if (fnv) fnv->add(p, n);
  return std::fwrite(p, 1, n, f) == n;
}

bool read_all(FILE* f, Fnv* fnv, void* p, size_t n) {
  if (std::fread(p, 1, n, f) != n) return false;
  if (fnv) fnv->add(p, n);
  return true;
}

struct CkptHeader {
  int32_t L[3], boundary, Q;
  double c[5];
  int32_t chi, precision;
  uint64_t seed;
  int32_t n_nodes;
};

bool read_header(FILE* f, Fnv* fnv, CkptHeader* h) {
  char tag[8];
  if (!read_all(f, fnv, tag, 8) || std::memcmp(tag, kCkptTag, 8) != 0) return false;
  return read_all(f, fnv, h->L, sizeof(h->L)) && read_all(f, fnv, &h->boundary, 4) && read_all(f, fnv, &h->Q, 4) &&
         read_all(f, fnv, h->c, sizeof(h->c)) && read_all(f, fnv, &h->chi, 4) &&
         read_all(f, fnv, &h->precision, 4) && read_all(f, fnv, &h->seed, 8) && read_all(f, fnv, &h->n_nodes, 4);
}
}  // namespace

QED_API int ttn_save(ttn_state* s, const char* path) {
  if (!s || !path) return fail(QED_EINVAL, "null argument");
  QED_TRY(
    qed::Engine* e = s->engine;
    int rc = e->move_to(e->n_nodes() - 1);
    if (rc) return engine_status(e, rc);
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(QED_EINVAL, "cannot open the checkpoint file for writing");
    Fnv fnv;
    const qed::Params& p = e->params();   // couplings as last set on the state
    const int32_t L[3] = {p.Lx, p.Ly, p.Lz};
    const double c[5] = {p.t, p.m, p.ge2, p.cB, p.nu};
    const int32_t chi = e->chi(), prec = e->precision(), nn = e->n_nodes();
    const uint64_t seed = e->seed();
    bool ok = write_all(f, &fnv, kCkptTag, 8) && write_all(f, &fnv, L, sizeof(L)) &&
              write_all(f, &fnv, &p.boundary, 4) && write_all(f, &fnv, &p.Q, 4) && write_all(f, &fnv, c, sizeof(c)) &&
              write_all(f, &fnv, &chi, 4) && write_all(f, &fnv, &prec, 4) && write_all(f, &fnv, &seed, 8) &&
              write_all(f, &fnv, &nn, 4);
    for (int i = 0; ok && i < nn; ++i) {
      const int64_t n = e->node_size(i);
      ok = write_all(f, &fnv, &n, 8);
    }
    std::vector<double> buf;
    for (int i = 0; ok && i < nn; ++i) {
      rc = e->node_export(i, &buf);
      if (rc) { std::fclose(f); return engine_status(e, rc); }
      ok = write_all(f, &fnv, buf.data(), buf.size() * sizeof(double));
    }
    ok = ok && write_all(f, nullptr, &fnv.h, 8);
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return fail(QED_EINVAL, "checkpoint write failed");
    return QED_OK;
  )
}

QED_API int ttn_load(const qed_model* m, const char* path, void* cuda_stream, ttn_state** out) {
  if (!m || !path || !out) return fail(QED_EINVAL, "null argument");
  *out = nullptr;
  QED_TRY(
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(QED_EINVAL, "cannot open the checkpoint file");
    Fnv fnv;
    CkptHeader h;
    if (!read_header(f, &fnv, &h)) { std::fclose(f); return fail(QED_EINVAL, "not a checkpoint file"); }
    const qed::Params& p = m->p;
    const double c[5] = {p.t, p.m, p.ge2, p.cB, p.nu};
    if (h.L[0] != p.Lx || h.L[1] != p.Ly || h.L[2] != p.Lz || h.boundary != p.boundary || h.Q != p.Q ||
        std::memcmp(h.c, c, sizeof(c)) != 0 || h.n_nodes != (int32_t)m->nodes.size()) {
      std::fclose(f);
      return fail(QED_EINVAL, "checkpoint parameters differ from the model");
    }
    // node sizes the model implies at the stored bond dimension: every size
    // read from the file must equal its expected value before anything is
    // allocated for it (a corrupt size cannot trigger a huge allocation)
    if (h.chi < 1 || h.chi > 4096) { std::fclose(f); return fail(QED_EINVAL, "checkpoint bond dimension out of range"); }
    std::vector<int64_t> expect;
    {
      std::vector<qed::Sectors> bonds;
      std::string err;
      if (!qed::sector_table(p, h.chi, m->nodes, &bonds, &err)) { std::fclose(f); return fail(QED_EINVAL, err.c_str()); }
      qed::Lattice lat{p.Lx, p.Ly, p.Lz, p.boundary == 1};
      for (const qed::TreeNode& nd : m->nodes) {
        qed::Sectors legs[2];
        for (int c = 0; c < 2; ++c)
          legs[c] = nd.child_kind[c] == 0 ? qed::physical_sectors(lat.parity(nd.child[c])) : bonds[nd.child[c]];
        const qed::Sectors& par = bonds[nd.index];
        int64_t size = 0;
        for (size_t ic = 0; ic < par.q.size(); ++ic)
          for (size_t ia = 0; ia < legs[0].q.size(); ++ia) {
            const int ib = legs[1].find(par.q[ic] - legs[0].q[ia]);
            if (ib >= 0) size += (int64_t)legs[0].dim[ia] * legs[1].dim[ib] * par.dim[ic];
          }
        expect.push_back(size);
      }
    }
    std::vector<int64_t> sizes(h.n_nodes);
    bool ok = true;
    for (int i = 0; ok && i < h.n_nodes; ++i) ok = read_all(f, &fnv, &sizes[i], 8) && sizes[i] == expect[i];
    if (!ok) { std::fclose(f); return fail(QED_EINVAL, "checkpoint node sizes differ from the model's layout"); }
    std::vector<std::vector<double>> data(h.n_nodes);
    for (int i = 0; ok && i < h.n_nodes; ++i) {
      data[i].resize(sizes[i]);
      ok = read_all(f, &fnv, data[i].data(), sizes[i] * sizeof(double));
    }
    uint64_t stored = 0;
    ok = ok && read_all(f, nullptr, &stored, 8) && stored == fnv.h;
    std::fclose(f);
    if (!ok) return fail(QED_EINVAL, "checkpoint truncated or corrupt");
    ttn_state* s = nullptr;
    int rc = ttn_create(m, h.chi, h.seed, h.precision, cuda_stream, &s);
    if (rc) return rc;
    std::vector<const double*> ptrs(h.n_nodes);
    for (int i = 0; i < h.n_nodes; ++i) ptrs[i] = data[i].data();
    rc = ttn_load_tensors(s, ptrs.data(), sizes.data(), h.n_nodes);
    if (rc) { ttn_destroy(s); return rc; }
    *out = s;
    return QED_OK;
  )
}

QED_API int ttn_apply_heff_adjoint_device(ttn_state* s, const double* x_device, double* y_device, int64_t n) {
  if (!s || !x_device || !y_device) return fail(QED_EINVAL, "null argument");
  if (n != s->engine->node_size(s->engine->center())) return fail(QED_EINVAL, "size must equal the centre tensor size");
  QED_TRY(return engine_status(s->engine, s->engine->apply_heff_adjoint(x_device, y_device));)
}

QED_API int ttn_energy_grad(ttn_state* s, int32_t node, const double* psi_device, int64_t n, double* energy,
                            double* dE_dpsi_device, double dE_dcoupling[5]) {
  if (!s || !dE_dcoupling) return fail(QED_EINVAL, "null argument");
  if (node >= s->engine->n_nodes()) return fail(QED_EINVAL, "node out of range");
  QED_TRY(
    if (node >= 0) {
      int rc = s->engine->move_to(node);
      if (rc) return engine_status(s->engine, rc);
    }
    if (psi_device && n != s->engine->node_size(s->engine->center()))
      return fail(QED_EINVAL, "size must equal the centre tensor size");
    if (dE_dpsi_device && n != s->engine->node_size(s->engine->center()))
      return fail(QED_EINVAL, "size must equal the centre tensor size");
    double e = 0.0;
    double dc[qed::N_CLASSES];
    int rc = s->engine->energy_grad(psi_device, &e, dE_dpsi_device, dc);
    for (int c = 0; c < qed::N_COUPLINGS; ++c) dE_dcoupling[c] = dc[c];
    if (rc) return engine_status(s->engine, rc);
    if (energy) *energy = e;
    return QED_OK;
  )
}

QED_API int ttn_gradient_step(ttn_state* s, double eta, double* e_before, double* e_after) {
  if (!s) return fail(QED_EINVAL, "null argument");
  if (!std::isfinite(eta)) return fail(QED_EINVAL, "eta must be finite");
  QED_TRY(return engine_status(s->engine, s->engine->gradient_step(eta, e_before, e_after));)
}

}  // extern "C"
