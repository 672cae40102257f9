// TTN sweep engine: device-resident U(1) block tensors, renormalized bond
// operators, H_eff plans, Lanczos eigensolver and isometry-centre moves.
#pragma once
#include <cuda_runtime.h>

#include <functional>
#include <map>
#include <memory>
#include <stdexcept>
#include <string>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "kernels.cuh"
#include "model.h"

namespace qed {

constexpr int kMaxKrylov = 128;   // largest Lanczos basis

// A device allocation that failed (reported as QED_ENOMEM at the C ABI).
struct DeviceAllocError : std::runtime_error {
  explicit DeviceAllocError(const std::string& what) : std::runtime_error(what) {}
};
// cudaMalloc that throws DeviceAllocError instead of returning an error code.
void device_alloc(void** p, size_t bytes, const char* what);

enum Precision { PREC_FP64 = 0, PREC_TF32 = 1, PREC_BF16 = 2, PREC_TF32X3 = 3 };

// Block layout of a three-leg tensor T[a, b, c] whose blocks (q_a, q_b)
// satisfy q_c = q_a + q_b - shift.  Blocks are ordered by (c-sector, q_a);
// inside a block elements are row-major (a, b, c).  The blocks of one
// c-sector therefore form a contiguous (rows x dim_c) row-major matrix.
struct Layout {
  Sectors leg[3];
  int shift = 0;
  struct Blk {
    int ia, ib, ic;
    int da, db, dc;
    long long off;       // element offset of the block
    int row0;            // first row of the block inside its c-sector matrix
  };
  std::vector<Blk> blk;
  std::map<std::pair<int, int>, int> index;
  std::vector<long long> sec_off;   // per c-sector: offset of its matrix
  std::vector<int> sec_rows;        // per c-sector: number of rows
  long long size = 0;
  void build(const Sectors& a, const Sectors& b, const Sectors& c, int shift_);
  int find(int ia, int ib) const {
    auto it = index.find({ia, ib});
    return it == index.end() ? -1 : it->second;
  }
};

// Host list of grouped-GEMM work plus its device copy.
// Outputs that name the same destination (pointer and shape) are merged, so
// every output region is written by exactly one output: contributions to a
// shared block are K-concatenated chunks, never concurrent writes.
// One tile-shape cut of a plan: tiles, chunks split into K parts where
// needed, outputs with their partial-sum slots, reduction list.
struct KVariant {
  std::vector<KTile> tiles;
  std::vector<KChunk> chunks;
  std::vector<KOutput> outs;
  std::vector<int> red;
  long long scratch_need = 0;
  KChunk* d_chunks = nullptr;
  KOutput* d_outs = nullptr;
  KTile* d_tiles = nullptr;
  int* d_red = nullptr;
  size_t cap_chunks = 0, cap_outs = 0, cap_tiles = 0, cap_red = 0;
  bool ready = false;
  void upload(cudaStream_t s);
  void release();
  ~KVariant() { release(); }
};

// Grouped-GEMM work list: outputs, each with its chunks (built through
// add_output / add_chunk, flattened by finalize), cut into tiles per tile
// shape on demand, with the chosen shape per arithmetic (FP64, FP32).
struct KPlan {
  std::vector<KChunk> chunks;
  std::vector<KOutput> outs;
  std::vector<std::vector<KChunk>> out_chunks;
  std::map<std::tuple<uintptr_t, long long, long long, int, int>, int> out_index;
  int current = -1;
  long long k_part = 4096;
  double flops = 0.0;   // 2 M N K over the GEMM chunks (set by finalize)
  KVariant var[KS_COUNT];
  int shape[3] = {-1, -1, -1};    // tuned tile shape per arithmetic (FP64, FP32, float-float), -1 while tuning
  int trials[3] = {0, 0, 0};
  cudaEvent_t tev[3][KS_COUNT][2][2] = {};   // [arithmetic][shape][repeat][start, stop]
  void clear() {
    chunks.clear(); outs.clear(); out_chunks.clear(); out_index.clear(); current = -1; flops = 0.0;
    for (KVariant& v : var) v.ready = false;
  }
  int add_output(double* C, long long c_m, long long c_n, int M, int N, int accumulate);
  void add_chunk(const KChunk& c);
  void finalize(long long k_part);
  KVariant& variant(int shape, cudaStream_t s);
  double padded_work(int shape) const;
  int candidates(int* out) const;
  void release();
  ~KPlan() { release(); }
};

// A dense renormalized operator on a bond: O[i', i] (row-major dim x dim)
// with charge-label shift q(i') - q(i) = shift.
struct BondOp {
  double* ptr = nullptr;
  int shift = 0;
};

struct BondOps {
  std::unordered_map<int, BondOp> term;
  double* H[N_CLASSES] = {};
  double* Htot = nullptr;
};

// One H_eff term at the centre: coef * op0 (x) op1 (x) op2.
// Bottom legs: site op of a term (row maps); bond legs: dense operators.
struct OpRef {
  int kind = 0;           // 0 = identity, 1 = bond operator, 2 = site term op (bottom leg)
  const double* ptr = nullptr;
  int shift = 0;
  int term = -1;          // for kind 2: the term whose site op acts here (-1: site Hamiltonian)
  int cls = -1;           // for kind 2 with term = -1: class of the site Hamiltonian (-1 = all)
};

struct HTerm {
  double coef = 1.0;
  int cls = -1;           // -1 = mixed (block Hamiltonians), else the coupling class
  OpRef op[3];
};

struct RowMap {
  int* map = nullptr;     // per output row, sign-encoded source row
  double* val = nullptr;  // optional per-row factor
  int src_sector = -1;    // source c-sector index (-1: all rows zero)
  long long nnz = 0;      // rows with a nonzero entry
};

// Mixed-precision H_eff plan of a bottom node (tensor-core kernel).
struct TcPlan {
  std::vector<TcTile> tiles;
  std::vector<TcOutput> outs;
  std::vector<TcChunk> chunks;
  std::vector<TcAdd> adds;
  std::vector<ConvJob> xjobs, wjobs;
  TcTile* d_tiles = nullptr;
  TcOutput* d_outs = nullptr;
  TcChunk* d_chunks = nullptr;
  TcAdd* d_adds = nullptr;
  ConvJob* d_xjobs = nullptr;
  ConvJob* d_wjobs = nullptr;
  size_t cap[6] = {0, 0, 0, 0, 0, 0};
  long long x_max_elems = 0, w_max_elems = 0;
  int max_kpad = 16, max_npad = 16;
  double flops_alg = 0, flops_exec = 0, bytes_alg = 0;
  long long wtot = 0;            // elements of the W buffer this plan uses
  void clear() {
    tiles.clear(); outs.clear(); chunks.clear(); adds.clear(); xjobs.clear(); wjobs.clear();
    x_max_elems = w_max_elems = wtot = 0; max_kpad = max_npad = 16; flops_alg = flops_exec = bytes_alg = 0;
  }
  void release();
  ~TcPlan() { release(); }
};

// Tensor-core leg-contraction plan (one launch of launch_tg_gemm).
struct TgPlan {
  std::vector<TgTile> tiles;
  std::vector<TgOut> outs;
  std::vector<TgChunk> chunks;
  std::vector<int> red;
  TgTile* d_tiles = nullptr;
  TgOut* d_outs = nullptr;
  TgChunk* d_chunks = nullptr;
  int* d_red = nullptr;
  size_t cap[4] = {0, 0, 0, 0};
  long long scratch_need = 0;   // floats of split-K partial sums
  int max_npad = 16;
  double flops = 0.0;           // algorithmic: 2 rows N K over the non-identity chunks
  void upload(cudaStream_t s);
  void release();
  ~TgPlan() { release(); }
};

// Digit-plane (FP64-accurate tensor-core) operator update of a bottom node.
struct OzPlan {
  std::vector<OzTile> tiles;
  std::vector<OzJob> jobs;
  std::vector<OzOut> outs;
  std::vector<OzSum> sums;
  OzTile* d_tiles = nullptr;
  OzJob* d_jobs = nullptr;
  OzOut* d_outs = nullptr;
  OzSum* d_sums = nullptr;
  size_t cap[4] = {0, 0, 0, 0};
  long long partial_elems = 0;
  int npad = 32;
  double flops = 0.0;   // algorithmic: 2 x mapped rows x chi_out x chi_in per job
  std::vector<void*> owned;   // row selections of the site Hamiltonians (engine allocations)
  void release();
  ~OzPlan() { release(); }
};

// Per kernel-class timing of launches on the engine stream (CUDA events).
// SIMT classes run FP64, or FP32 inside the low-precision phase of a mixed state.
// KC_MOVE and KC_LANCZOS time whole phases (centre moves with QR and
// operator updates; Lanczos calls including their products).
enum KernelClass {
  KC_TC_HEFF = 0, KC_HEFF_SIMT_BOTTOM = 1, KC_HEFF_SIMT_UPPER = 2, KC_MOVE = 3, KC_LANCZOS = 4,
  KC_MOVE_QR = 5,    // per bond: QR of the departing tensor and R absorption (FP64)
  KC_MOVE_OPS = 6,   // per bond: renormalized / environment operator update at an upper node
  KC_MOVE_OPS_BOTTOM = 7,   // per bond: operator update leaving a bottom node upwards
  KC_COUNT = 8
};
struct KernelTiming {
  double ms = 0.0;
  long long launches = 0;
  double flops_alg = 0.0;
  double flops_exec = 0.0;
  double bytes_alg = 0.0;
};

struct SweepStats {
  double energy = 0.0;
  int matvecs = 0;
  int matvecs_mixed = 0;
  int node_updates = 0;
  double max_residual = 0.0;
  int not_converged = 0;
};

class Engine {
 public:
  Engine(const Params& p, int chi, uint64_t seed, int precision, cudaStream_t stream);
  ~Engine();

  // One full sweep (nodes in sweep_order); energies[i] per node update.
  int sweep(double tol, int max_krylov, SweepStats* st, std::vector<double>* energies);
  // Energy with the current centre tensor; class-resolved parts.
  int energy(double* total, double parts[N_CLASSES]);
  // Single-site diagonal probabilities (267 per site), centre moved to the root.
  int site_probabilities(std::vector<double>* probs);
  int node_export(int node, std::vector<double>* host);
  int node_import(int node, const std::vector<double>& host);
  // Replace every tensor (tree isometric towards the root, root normalised)
  // and rebuild all renormalized operators; the centre becomes the root.
  int load_tensors(const double* const* host, const long long* sizes, int n);
  // New coupling constants (t, m, ge2, cB, nu) on the same lattice and
  // charge sector: the term coefficients are replaced (the same expressions
  // as at creation), every cached plan or row map that holds a coefficient
  // is dropped and freed, and all renormalized operators are rebuilt from
  // the current tensors; the centre becomes the root.  A coupling class that
  // was zero at creation has no terms and cannot be switched on (-1).
  int set_couplings(const Params& np);
  const Params& params() const { return p_; }
  int move_to(int target);
  // Work list of y = H_eff x at a bottom-node centre for the FP64 grouped
  // GEMM, written into caller-provided arrays with no allocation: x and y
  // are used in place, row maps and environment operators must already
  // exist.  Returns 0, -7 if the centre is not a bottom node or a needed
  // row map is missing, -2 if an array is too small.
  int noalloc_worklist(const double* x, double* y, KTile* tiles, int max_tiles, KOutput* outs, int max_outs,
                       KChunk* chunks, int max_chunks, int* n_tiles, int* n_outs, int* n_chunks);
  int optimize_node(int node, double tol, int max_krylov, SweepStats* st, double* e);
  // H_eff x at the current centre (x, y device pointers, centre layout).
  int apply_heff(const double* x, double* y, int cls_filter);
  // y = H_eff^T x (transposed terms, FP64) at the current centre.
  int apply_heff_adjoint(const double* x, double* y);
  // Energy, dE/dpsi (device, optional) and dE/dcoupling[5] at the centre for
  // psi (device, centre layout) or the centre tensor when psi == nullptr.
  int energy_grad(const double* psi, double* energy, double* grad, double dc[N_CLASSES]);
  // psi <- normalize(psi - eta dE/dpsi) on the centre tensor.
  int gradient_step(double eta, double* e_before, double* e_after);
  // H_eff x in the state's precision (tensor cores at bottom nodes when mixed)
  int apply_heff_native(const double* x, double* y) {
    use_mixed_ = precision_ != PREC_FP64;
    int rc = apply_heff(x, y, -1);
    use_mixed_ = false;
    return rc;
  }
  long long node_size(int node) const { return layout_[node].size; }
  int center() const { return center_; }
  int n_nodes() const { return (int)nodes_.size(); }
  const std::vector<Sectors>& bonds() const { return bonds_; }
  const Layout& layout(int n) const { return layout_[n]; }
  double constant() const { return constant_; }
  int n_terms() const { return (int)terms_.size(); }
  cudaStream_t stream() const { return stream_; }
  double* tensor(int n) { return T_[n]; }
  const std::string& error() const { return err_; }
  long long device_bytes() const { return bytes_; }
  int last_lanczos_iters = 0;
  int last_mixed_iters = 0;
  double last_residual = 0.0;
  // low-precision phase of the last mixed update: Ritz value and relative
  // residual before the FP64 correction (NaN after an FP64 update)
  double last_mixed_ritz = 0.0;
  double last_mixed_residual = 0.0;
  // kernel timing (enabled by set_profiling): resolved on read
  void set_profiling(bool on);
  int kernel_timing(KernelTiming out[KC_COUNT]);
  void reset_timing();
  int precision() const { return precision_; }
  int chi() const { return chi_; }
  uint64_t seed() const { return seed_; }
  void set_precision(int p);
  // mixed path tuning: residual target of the low-precision phase
  double mixed_tol = 0.0;
  // bound of each mbarrier wait of the tensor-core kernels, in polls (< 0: default)
  long long wait_polls = -1;

 private:
  Params p_;
  int chi_;
  uint64_t seed_;
  int precision_;
  cudaStream_t stream_;
  Lattice lat_;
  std::vector<Term> terms_;
  double constant_ = 0.0;
  std::vector<TreeNode> nodes_;
  std::vector<Sectors> bonds_;
  std::vector<Layout> layout_;
  std::vector<std::vector<char>> in_region_;
  std::vector<double*> T_;
  std::vector<BondOps> up_, down_;
  int center_ = -1;
  std::string err_;
  long long bytes_ = 0;
  std::vector<void*> allocs_;
  std::map<long long, SiteOp*> site_ops_;   // packed (parity, kind, a, b)
  // row maps of bottom nodes: (node, term) -> per output c-sector
  std::map<std::pair<int, int>, std::vector<RowMap>> rowmaps_;
  double* zpool_ = nullptr;
  long long zpool_elems_ = 0;
  double* x_in_ = nullptr;
  double* y_out_ = nullptr;
  double* tmp_ = nullptr;
  double* scratch_ = nullptr;
  long long scratch_elems_ = 0;
  KPlan work_;
  // Plans are built once per (kind, node, ...) and replayed: their device
  // pointers (tensors, bond operators, fixed buffers, Z pool) are stable
  // until the Z pool or the staging buffers are reallocated, which clears
  // the caches.  Split-K scratch is passed at launch, not stored.
  std::map<std::tuple<int, int, int, int>, std::unique_ptr<KPlan>> plan_cache_;
  KPlan* cached_plan(int kind, int a, int b, int c, const std::function<void(KPlan&)>& build);
  int launch_plan(KPlan* pl, int fp32 = 0);
  int launch_kplan(KPlan& pl, int fp32, bool tune);
  int forced_shape_ = -1;   // QED_KC_SHAPE
  double ops_flops_ = 0.0;   // flops of the plans launched since the last reset (profiling)
  void clear_plan_caches();
  // three-stage plans (Z stages of upper nodes, then the output stage)
  void cached_plans(int kind, int a, int b, int n, KPlan** out, const std::function<void(KPlan**)>& build);
  struct HeffPlans {
    KPlan st[3];
    long long z_elems = 0;       // Z pool prefix the stages use
    double flops = 0.0;          // algorithmic flops of one product
  };
  std::map<std::pair<int, int>, std::unique_ptr<HeffPlans>> heff_cache_;
  HeffPlans* heff_plans(int node, int cls_filter, bool adjoint);
  std::map<const int*, RowMap> inv_maps_;   // inverse row maps of the adjoint
  const RowMap& inverse_rowmap(const RowMap& fwd, int rows_fwd, int rows_inv);
  double* grad_a_ = nullptr;
  double* grad_b_ = nullptr;
  double* grad_c_ = nullptr;
  // persistent QR / move buffers (largest bond dimension squared)
  double* qr_G_ = nullptr;
  double* qr_Rinv_ = nullptr;
  double* qr_Racc_ = nullptr;
  double* qr_Rtmp_ = nullptr;
  double* move_R_ = nullptr;
  struct QrDesc {
    long long* off = nullptr;
    int* n = nullptr;
    int* ld = nullptr;
    int* status = nullptr;
    int count = 0;
    int max_n = 0;
  };
  std::map<std::pair<int, int>, QrDesc> qr_desc_;
  // mixed-precision state: per-node plans; the staging buffers are shared
  // and the environment blocks are re-staged when the centre changes
  std::map<int, std::unique_ptr<TcPlan>> tc_cache_;
  // mixed-precision upper-node products on the tensor cores: three stages
  // per node (first child leg, second child leg, parent leg with the sum over
  // terms); FP32 intermediates in tg_pool_, identity blocks in ident_
  struct TgHeff {
    TgPlan st[3];
    double flops = 0.0;
  };
  std::map<int, std::unique_ptr<TgHeff>> tg_cache_;
  float* tg_pool_ = nullptr;
  long long tg_pool_elems_ = 0;
  float* tg_scratch_ = nullptr;
  long long tg_scratch_elems_ = 0;
  double* ident_ = nullptr;
  int ident_dim_ = 0;
  TgHeff* tg_plans(int node);
  std::map<int, std::unique_ptr<OzPlan>> oz_cache_;
  void* oz_planes_ = nullptr;
  double* oz_partial_ = nullptr;
  long long oz_partial_elems_ = 0;
  int compute_up_oz(int node, const std::vector<std::pair<double*, double>>& terms, const std::vector<int>& keys,
                    BondOps& out);
  int apply_heff_tg();
  int tc_w_node_ = -1;          // node whose environment blocks are staged
  void clear_tc_cache();
  void* xstage_ = nullptr;      // BF16 or FP32 padded staging of x
  float* xstage32_ = nullptr;   // FP32 padded staging (BF16 path)
  long long xstage_elems_ = 0;
  void* wbuf_ = nullptr;
  long long wbuf_elems_ = 0;
  int* d_err_ = nullptr;
  bool profiling_ = false;
  struct EvRec { cudaEvent_t a, b; int cls; double fa, fe, ba; };
  std::vector<EvRec> ev_pending_;
  std::vector<cudaEvent_t> ev_pool_;
  KernelTiming timing_[KC_COUNT];
  cudaEvent_t ev_get();
  void ev_begin(cudaEvent_t* e);
  void ev_end(cudaEvent_t a, int cls, double fa, double fe, double ba);
  TcPlan* tc_plan(int node);
  TcPlan* tc_prepare();
  // bumped whenever cached plans are dropped (their device pointers go stale)
  uint64_t gen_ = 0;
  int apply_heff_mixed();
  bool mixed_node(int node) const;
  // Lanczos workspace
  double* V_ = nullptr;
  double* zb_ = nullptr;        // rotated Ritz vectors of a thick restart
  // side stream for the per-iteration tridiagonal solve and its readback
  cudaStream_t aux_ = nullptr;
  cudaEvent_t ev_iter_[129] = {};
  cudaEvent_t ev_conv_[129] = {};
  double* ring_dev_ = nullptr;    // 4 doubles per iteration: theta, residual
  double* ring_host_ = nullptr;   // pinned copy: theta, residual, beta
  int last_conv_ = -1;
  long long zb_elems_ = 0;
  int kmax_alloc_ = 0;
  double* d_scal_ = nullptr;   // alpha[128], beta[128], s[128], out[8], coeffs[128], partials
  double* d_partial_ = nullptr;
  long long nmax_ = 0;

  // device allocations (base, bytes) for the optional plan validator
  std::map<uintptr_t, size_t> ranges_;
  bool validate_ = false;
  bool validate_plan(const KPlan& pl, const KVariant& v, const char* what);
  void track(void* p, size_t bytes) { if (p) ranges_[(uintptr_t)p] = bytes; }
  void untrack(void* p) { ranges_.erase((uintptr_t)p); }
  bool in_range(const void* p, long long lo_off, long long hi_off) const;   // own or a peer's
  bool in_own_range(const void* p, long long lo_off, long long hi_off) const;
  std::vector<const Engine*> peers_;   // other engines whose allocations a grouped plan may touch
  void* dalloc(size_t bytes);
  // free allocations made by dalloc (null entries ignored)
  void dfree_all(const std::vector<void*>& ptrs);
  bool check(cudaError_t e, const char* what);
  const SiteOp* site_op(int parity, const OpKey& key);
  bool touches(int term, int node) const;
  bool touches_sites(int term, const std::vector<char>& reg) const;
  bool inside(int term, int node) const;
  bool crosses(int term, int node) const;
  int leg_node(int node, int leg) const;  // child node id or -1 for a site
  int leg_site(int node, int leg) const;
  const Sectors& leg_sectors(int node, int leg) const;
  void init_tensors();
  int qr_toward(int node, int leg, double* Rout);
  int qr_gram_schmidt(int node, int leg, double* Rout);
  int absorb(int node, int leg, const double* R);
  int compute_up(int node);
  int compute_down(int node);
  const std::vector<RowMap>& rowmap(int node, int term);
  RowMap build_rowmap_sector(int node, const SiteOp* A, const SiteOp* B, int out_sector, const std::vector<double>* vals);
  const std::vector<RowMap>& site_ham_map(int node, int leg, int cls);
  void build_heff_terms(int node, int cls_filter, std::vector<HTerm>* out);
  int run_plan(KPlan& pl);
  void plan_leg_apply(KPlan& pl, const Layout& LX, const double* X, const Layout& LY, double* Y, int leg,
                      const double* P, int dimP, int shiftP, bool transposed, double alpha);
  void plan_contract_but(KPlan& pl, const Layout& LT, const double* T, const Layout& LZ, const double* Z, int leg,
                         double* O, int dimO, double alpha);
  void ensure_scratch(long long elems);
  void ensure_zpool(long long elems);
  Layout shifted(int node, int shift) const;
  int lanczos(int node, double tol, int max_krylov, bool mixed, int max_restarts, double* energy, double* resid,
              int* iters);
  int lanczos_run(int node, double tol, int max_krylov, bool mixed, int max_restarts, double* energy, double* resid,
                  int* iters);
  int move_path(int target);
  // Lanczos building blocks
  int lz_prepare(int kmax);
  void lz_start(int node);
  void lz_iteration(int j, long long n);
  void lz_next_vector(int j, long long n);
  int lz_thick_restart(int k, int kmax, long long n, int* j0);
  void lz_finish(int node, int k);
  void lz_queue_check(int j);
  bool lz_converged(int slot, double tol, double* theta, double* res) const;
  friend class BatchRunner;
  bool use_mixed_ = false;   // current matvec precision inside lanczos
  // products of a mixed state's FP64 residual correction run in float-float
  // arithmetic (FP64-level accuracy on the FP32 pipes)
  bool ff_products_ = false;
  int ops_mode() const { return precision_ != PREC_FP64 ? 2 : 0; }
};

}  // namespace qed
