/*
 * qedttn: GB300 (sm_103a) hot path of the Tree Tensor Network ground-state
 * search for compact (3+1)D lattice QED of Magnifico, Felser, Silvi and
 * Montangero, "Lattice Quantum Electrodynamics in (3+1)-dimensions at finite
 * density with Tensor Networks" (arXiv:2011.10658).
 *
 * The library builds the problem the paper states -- the gauge-invariant
 * dressed-site basis (Methods, Eq. (12)-(14)), the Hamiltonian of Eq. (1)
 * written as products of local operators (Eq. (15) and the plaquette
 * factorisation) plus the link penalty of Eq. (16), in a fixed total-charge
 * sector -- and sweeps a U(1)-symmetric binary TTN (Methods, "Tensor
 * Networks": H_eff of one tensor, its lowest eigenpair by a Krylov method,
 * tensor update, sweeping from the lowest to the highest layer).
 *
 * Conventions
 *  - Return value: a qed_status (0 = success, negative = error).  After an
 *    error, qed_last_error() returns a message (thread-local).
 *  - Opaque handles are owned by the library and freed by the *_destroy
 *    functions.  Output buffers are owned by the caller; sizes are counted in
 *    elements; passing a NULL buffer (or cap = 0) queries the size in *n.
 *  - Host pointers unless the name says "device".  The stream passed to
 *    ttn_create is used for every kernel of that state; calls that return
 *    host values synchronise that stream.  One state per thread at a time.
 *  - No C++ exception crosses this boundary.
 */
#ifndef QEDTTN_H
#define QEDTTN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Couplings and lattice of Eq. (1) + Eq. (16).  The couplings are taken as
 * independent inputs (Results, "The model": the numerical setup treats t, m,
 * g_e, g_m as mutually independent).  The plaquette term enters as
 * -cB * sum(box + h.c.), i.e. cB = g_m^2 / 2.  nu is the link-constraint
 * penalty of Eq. (16).  Q is the total charge sum_x (psi^dag psi -
 * (1 - (-1)^x)/2) (Eq. (1) text).  boundary: 0 = open, every site keeps its
 * six half-links and the ones pointing out of the lattice are free
 * ("dangling", each costing ge2/2 (1 - k)^2); 1 = periodic (Results,
 * "Transition at zero charge"): every direction with more than one site
 * wraps around, so its half-links all belong to links (on an extent of 2
 * two links join the same pair of sites), while a direction of extent 1
 * keeps open, dangling half-links.  Other values are rejected. */
typedef struct {
  int32_t Lx, Ly, Lz;
  int32_t boundary;
  double t, m, ge2, cB, nu;
  int32_t Q;
} qed_params;

typedef enum {
  QED_OK = 0,
  QED_EINVAL = -1,      /* invalid argument */
  QED_ENOMEM = -2,      /* device or host allocation failed */
  QED_ECUDA = -3,       /* CUDA runtime error */
  QED_ENOCONV = -4,     /* eigensolver stopped above tolerance; result valid */
  QED_ENAN = -5,        /* non-finite input or rank-deficient factorisation */
  QED_ETIMEOUT = -6,    /* a device wait hit its iteration limit */
  QED_EUNSUPPORTED = -7 /* configuration outside what this build supports */
} qed_status;

/* Arithmetic of the H_eff products inside the eigensolver (Lanczos vectors,
 * QR, operator updates and reported energies are FP64 in every mode):
 * FP64; TF32 or BF16 tensor-core operands with FP32 accumulation; TF32X3:
 * operands split as hi + lo TF32 parts, three products per term (about 21
 * significant bits).  Upper (non-bottom) nodes use FP32 arithmetic in the
 * mixed modes. */
enum { QED_PREC_FP64 = 0, QED_PREC_TF32 = 1, QED_PREC_BF16 = 2, QED_PREC_TF32X3 = 3 };

/* Local operator kinds of qed_local_op (half-link index j: 0..5 for
 * -x, -y, -z, +x, +y, +z). */
enum {
  QED_OP_IDENTITY = 0,
  QED_OP_M = 1,    /* psi^dag eta_j        (Eq. (15))          */
  QED_OP_MD = 2,   /* eta_j^dag psi        (Eq. (15))          */
  QED_OP_C = 3,    /* eta_i^dag eta_j      (plaquette factor)  */
  QED_OP_P = 4,    /* projector on k_j = k (Eq. (16))          */
  QED_OP_N = 5,    /* psi^dag psi          (mass term)         */
  QED_OP_E2 = 6,   /* sum over mask j of (1 - k_j)^2, Eq. (10) squared; j1 = bit mask */
  QED_OP_PC = 8    /* 1 - projector on k_j = k (penalty factor)                  */
};

typedef struct qed_model qed_model;
typedef struct ttn_state ttn_state;

/* Dressed-site basis of Eq. (12)-(14) for parity +1 (even) or -1 (odd).
 * table: [267][9] int8 rows (phi, k1..k6, sign of Eq. (12), charge q);
 * rows ordered phi outer, then (k1..k6) lexicographic.  NULL table: only
 * *n_rows is written.  Errors: QED_EINVAL for another parity. */
int qed_basis(int parity, int8_t *table, int32_t *n_rows);

/* Local operator in monomial form on a site of the given parity:
 * (O v)[i] = val[i] * v[src[i]], src[i] = -1 for a zero row.  src[267],
 * val[267] caller-owned.  For QED_OP_C, j1 = i and j2 = j; for QED_OP_P,
 * j1 = j and j2 = k; for QED_OP_E2, j1 = bit mask.  Built from the rishon
 * algebra of Eq. (6) with Jordan-Wigner signs inside the site. */
int qed_local_op(int parity, int op_kind, int j1, int j2, int16_t *src, double *val);

/* Model: lattice, product-term list of Eq. (1) + (16), binary tree (Methods,
 * "Tensor Networks": x-pairs, then y, then z, repeating).  Lattice extents
 * must be powers of two with at least two sites. */
int qed_model_create(const qed_params *p, qed_model **out);
void qed_model_destroy(qed_model *m);
/* Local chemical potentials (Methods, "Fermionic compact representation":
 * the diagonal local terms used to pin charges; Results, "Quantum
 * capacitor": large potentials on two opposite faces): one term
 * mu[x] psi^dag_x psi_x per site with mu[x] != 0, in a coupling class of
 * its own (class 5).  n = number of sites (caller-owned mu, copied), or
 * n = 0 to remove them.  Applies to states created from the model
 * afterwards.  QED_ENAN on a non-finite entry. */
int qed_model_set_site_potential(qed_model *m, const double *mu, int32_t n);
/* n_sites, number of product terms, number of tree nodes, additive constant
 * (zero: the penalty of Eq. (16) is written as nu sum_k P^k_x (1 -
 * P^{2-k}_y) per link, an exact rewrite of nu (1 - delta_{2,L})). */
int qed_model_info(const qed_model *m, int32_t *n_sites, int32_t *n_terms, int32_t *n_nodes, double *constant);
/* Term list: for term i, coef[i], cls[i] (0 t, 1 m, 2 ge2, 3 cB, 4 nu, 5 mu) and up
 * to four factors ops[i][f] = (site, kind, a, b) with n_ops[i] factors. */
int qed_model_terms(const qed_model *m, double *coef, int32_t *cls, int32_t *n_ops, int32_t *ops /* [n][4][4] */,
                    int64_t cap, int64_t *n);
/* Tree: per node (layer, axis, child_kind0, child0, child_kind1, child1,
 * parent); child_kind 0 = site, 1 = node; parent -1 for the root. */
int qed_model_tree(const qed_model *m, int32_t *nodes /* [n][7] */, int64_t cap, int64_t *n);
/* Order of the node updates in one sweep (Methods: the sweep runs from the
 * lowest to the highest layer; the order inside a layer is not given there).
 * Inside a layer: depth-first order of the tree, first child first, the
 * direction alternating between consecutive layers.  order[i] = node id;
 * *n = number of nodes.  Caller-owned buffer of cap entries (QED_EINVAL if
 * too small; a NULL buffer only reports *n). */
int qed_model_sweep_order(const qed_model *m, int32_t *order, int64_t cap, int64_t *n);
/* Bond sector table for bond dimension chi: for the bond above each node,
 * its sectors as consecutive (node, q, dim) triples. */
int qed_model_sectors(const qed_model *m, int32_t chi, int32_t *triples, int64_t cap, int64_t *n);

/* TTN state on the current CUDA device.  Tensors start as SplitMix64-seeded
 * random isometries (per-sector QR with positive diag R), the centre at the
 * root, all renormalized operators built.  precision: QED_PREC_*.
 * cuda_stream: a cudaStream_t (NULL = the legacy default stream). */
int ttn_create(const qed_model *m, int32_t chi, uint64_t seed, int precision, void *cuda_stream, ttn_state **out);
void ttn_destroy(ttn_state *s);

typedef struct {
  double energy;            /* last eigenvalue (penalty and constant included) */
  int32_t matvecs;          /* H_eff applications (all precisions) */
  int32_t matvecs_mixed;    /* of which on the tensor-core (TF32/BF16) path */
  int32_t node_updates;
  int32_t not_converged;    /* node updates that stopped above tolerance */
  double max_rel_residual;  /* max |beta_k s_k| / |theta| */
  double seconds;           /* wall time of the call */
} ttn_sweep_stats;

/* n_sweeps full sweeps: nodes in qed_model_sweep_order (layer by layer from
 * the bottom), the centre moved along the tree with per-sector QR, each node
 * replaced by the lowest eigenvector of its H_eff (Lanczos with full
 * reorthogonalisation, started from the current tensor, stopping at
 * residual <= tol |theta|, restarted every max_krylov steps).
 * Returns QED_ENOCONV (stats still valid) if some update stopped early. */
int ttn_sweep(ttn_state *s, int32_t n_sweeps, double tol, int32_t max_krylov, ttn_sweep_stats *out);
/* Mixed precision (QED_PREC_TF32 / QED_PREC_BF16): bottom-node updates run
 * Lanczos with tensor-core H_eff products until the residual reaches
 * max(0.3 tol, mixed_tol) (or stops improving), then continue from that Ritz
 * vector with FP64 products until the FP64 residual reaches tol.  Default
 * mixed_tol: 1e-7 (TF32X3), 1e-5 (TF32), 1e-4 (BF16). */
int ttn_set_mixed_tol(ttn_state *s, double mixed_tol);

/* New couplings {t, m, ge2, cB, nu} (the order of the coupling classes) for
 * the same lattice and charge sector.  Term coefficients become those a
 * model created with these couplings has; every renormalized operator is
 * rebuilt from the current tensors (no tensor changes) and the centre moves
 * to the root.  A class whose coupling was zero at creation has no terms and
 * cannot be switched on (QED_EINVAL); a class may be switched off (0).  Used
 * by the driven optimisation below, which changes nu between sweeps. */
int ttn_set_couplings(ttn_state *s, const double couplings[5]);

/* Driven optimisation (Methods, "Numerical Convergence", the paragraph on
 * the penalty of Eq. (16)) with the Lanczos tolerance raised each sweep
 * (Methods, "Tensor Networks": the eigensolver's precision grows from
 * sweep to sweep).  The penalty nu of sweep s:
 *   linear stage:    nu_0 = nu_start, nu_{s+1} = nu_s + nu_step, until the
 *                    energy <H + H_pen> after a sweep exceeds the previous
 *                    sweep's by more than rise_rel |E_prev| (a small
 *                    increase; rise_rel keeps rounding from counting),
 *                    which ends the stage;
 *   quadratic stage: nu = nu_switch + quad_coef * nu_step * k^2 for the k-th
 *                    sweep after the switch (k = 1, 2, ...; quad_coef < 1
 *                    makes the first increments smaller than nu_step);
 *   constant stage:  once a stage would pass nu_max, nu = nu_max for every
 *                    later sweep; the run has converged when, after at least
 *                    min_final_sweeps sweeps at nu_max, two consecutive
 *                    energies differ by <= conv_rel |E|.
 * The Lanczos tolerance of sweep s is max(tol_final, tol_start tol_factor^s).
 * The paper gives no numbers for any of these: they are inputs. */
typedef struct {
  double nu_start, nu_step, quad_coef, nu_max;
  double tol_start, tol_factor, tol_final;
  double conv_rel, rise_rel;
  int32_t min_final_sweeps; /* >= 2 */
  int32_t max_sweeps;
  int32_t max_krylov;
} qed_drive;

/* Schedule state: the stage (0 linear, 1 quadratic, 2 constant), the sweep
 * index, nu and tolerance of the next sweep, done = 1 once converged. */
typedef struct {
  int32_t stage, sweep, since_switch, final_sweeps, done;
  double nu, tol, nu_switch, e_prev;
} qed_drive_state;

/* Host-only schedule steps (no GPU): qed_drive_start sets nu and tol of
 * sweep 0; qed_drive_next takes the energy of the sweep just run and sets
 * those of the next one (or done).  QED_EINVAL on inconsistent settings
 * (nu_start <= 0, nu_step <= 0, nu_max < nu_start, quad_coef <= 0, tolerances
 * not positive, tol_factor outside (0, 1], conv_rel or rise_rel negative,
 * min_final_sweeps < 2). */
int qed_drive_start(const qed_drive *d, qed_drive_state *st);
int qed_drive_next(const qed_drive *d, qed_drive_state *st, double energy);

/* One record per sweep of ttn_drive. */
typedef struct {
  int32_t sweep, stage;
  double nu, tol;
  double energy;                 /* <H + H_pen> after the sweep */
  double energy_without_penalty; /* <H> */
  double delta_L;                /* sum over links |<L - 2>| (Methods, Numerical Convergence) */
  int32_t matvecs, not_converged;
  double max_rel_residual, seconds;
} qed_drive_record;

/* Run the driven optimisation on s from its current tensors: before each
 * sweep ttn_set_couplings with the schedule's nu (the other couplings as
 * the state has them), one sweep at the schedule's tolerance, then the
 * energies and delta_L.  Records go to log[0 .. min(n, cap)) (caller-owned;
 * NULL with cap 0 allowed); *n = sweeps run.  QED_OK once converged,
 * QED_ENOCONV if max_sweeps ran out first (records valid). */
int ttn_drive(ttn_state *s, const qed_drive *d, qed_drive_record *log, int32_t cap, int32_t *n);
/* Bound of every mbarrier wait inside the tensor-core kernels of this state,
 * in polls (each poll is one mbarrier test plus a 32 ns sleep); polls < 0
 * restores the default (2^22 polls, about a quarter of a second).  A wait
 * that runs out sets a device flag, the kernel drains the MMAs it issued,
 * frees its tensor memory and returns; the node update then returns
 * QED_ETIMEOUT and the state stays usable.  No counterpart in the paper: a
 * failure-detection control (polls = 0 makes every such wait give up at
 * once, which is how the tests reach that path without a GPU fault). */
int ttn_set_wait_limit(ttn_state *s, int64_t polls);
/* n_sweeps sweeps of n independent problems together (batching of
 * independent ground-state problems, e.g. several charge sectors and
 * couplings; the paper's finite-density results scan the charge Q, Results,
 * each value a separate ground-state search -- running several at once has
 * no counterpart there).  The states must share the lattice size, the precision and
 * the CUDA stream; sector tables, couplings and seeds may differ.  The
 * problems update each node together: per-problem centre moves, then a
 * lockstep Lanczos (same algorithm as ttn_sweep) whose H_eff products for
 * all problems are one grouped launch (the tensor-core tiles or grouped-GEMM
 * chunks of every problem), replayed from a CUDA graph once the grouped
 * GEMM's tile shape is tuned (no graph on the legacy default stream); the
 * FP64 check of a mixed-precision update runs per problem.  out: n entries
 * (seconds = wall time of the whole call).  QED_ENOCONV if some update of
 * some problem stopped above tolerance (stats valid). */
int ttn_batch_sweep(ttn_state *const *states, int32_t n, int32_t n_sweeps, double tol, int32_t max_krylov,
                    ttn_sweep_stats *out);
/* Switch the product precision of an existing state (QED_PREC_*); resets
 * mixed_tol to its default for that precision. */
int ttn_set_precision(ttn_state *s, int precision);
/* Last node update: FP64 and mixed Lanczos iterations, |beta s| / |theta|
 * of the final (FP64) Ritz pair, and for a mixed update the Ritz value and
 * relative residual that the low-precision phase reached before the FP64
 * correction (NaN after an FP64 update).  Any output may be NULL. */
int ttn_last_update(ttn_state *s, int32_t *iters_fp64, int32_t *iters_mixed, double *rel_residual,
                    double *ritz_mixed, double *rel_residual_mixed);

/* Kernel timing with CUDA events on the state's stream (off by default).
 * kernel_class: 0 = tensor-core bottom-node H_eff, 1 = SIMT bottom-node
 * H_eff (FP64), 2 = upper-node H_eff (FP64 SIMT, or tensor-core leg
 * contractions in the low-precision phase of a mixed state), 3 = whole
 * centre moves (QR, R absorption, operator updates), 4 = whole Lanczos calls
 * (products included; the difference is vector work and idle time), 5 =
 * per-bond QR and R absorption of a move, 6 = per-bond operator update at an
 * upper node (FP64; flops = its grouped-GEMM chunks), 7 = per-bond operator
 * update leaving a bottom node upwards (FP64, or FP64-accurate digit-plane
 * products on the tensor cores in a mixed state; flops = 2 x mapped rows x
 * chi_out x chi_in per term and sector).  Returns accumulated milliseconds,
 * launches, algorithmic flops (nonzero rows of the monomial gathers times
 * the dense environment contraction), executed flops (padded tiles) and
 * algorithmic bytes (staged input read, FP64 output written, operator
 * blocks read) since the last reset. */
int ttn_set_profiling(ttn_state *s, int on);
int ttn_reset_timing(ttn_state *s);
int ttn_kernel_timing(ttn_state *s, int kernel_class, double *ms, int64_t *launches, double *flops_alg,
                      double *flops_exec, double *bytes_alg);

/* Optimise one node (moving the centre there first). */
int ttn_optimize_node(ttn_state *s, int32_t node, double tol, int32_t max_krylov, double *energy);
/* Move the isometry centre to a node. */
int ttn_move_center(ttn_state *s, int32_t node);
int ttn_info(ttn_state *s, int32_t *center, int32_t *n_nodes, int64_t *max_node_size);
int ttn_node_size(ttn_state *s, int32_t node, int64_t *n);

/* <H + H_pen> of the state (constant included) and the same without the
 * penalty; E_class[5] (nullable) = <H_class> per coupling class t, m, ge2,
 * cB, nu (constant in the nu class), i.e. dE/dc_class times c_class.  The
 * chemical-potential energy (class 5) is E_total minus the sum of these. */
int ttn_energy(ttn_state *s, double *E_total, double *E_without_penalty, double *E_class);

/* Observables (Results text and Eq. (16a), (17b)), centre moved to the root:
 *  QED_MEAS_PROBS  : [N_sites][267] diagonal of each single-site reduced
 *                    density matrix
 *  QED_MEAS_PHI    : [N_sites] <psi^dag psi>
 *  QED_MEAS_NX     : [N_sites] n_x = (1 + p)/2 - p <psi^dag psi>
 *  QED_MEAS_QX     : [N_sites] <q_x>
 *  QED_MEAS_K      : [N_sites][6] <k_j>
 *  QED_MEAS_ELINK  : [N_links] <E> on each internal link (Eq. (10))
 *  QED_MEAS_SCALARS: [4] rho, delta_L, sum_x <q_x>, number of sigma layers
 *  QED_MEAS_SIGMA  : [layers] sigma(l), l = 1.. distance to the boundary */
enum {
  QED_MEAS_PROBS = 0, QED_MEAS_PHI = 1, QED_MEAS_NX = 2, QED_MEAS_QX = 3, QED_MEAS_K = 4,
  QED_MEAS_ELINK = 5, QED_MEAS_SCALARS = 6, QED_MEAS_SIGMA = 7
};
int ttn_measure(ttn_state *s, int kind, double *out, int64_t cap, int64_t *n);

/* Copy of one node tensor in its block layout (FP64): blocks ordered by
 * (parent sector, left charge), each block row-major (left, right, parent). */
int ttn_node_export(ttn_state *s, int32_t node, double *buf, int64_t cap, int64_t *n);
/* Replace one node tensor (same layout).  QED_ENAN on non-finite input. */
int ttn_node_import(ttn_state *s, int32_t node, const double *buf, int64_t n);
/* Resume from host-held tensors: bufs[i] (sizes[i] elements, block layout)
 * for every node i; the tree must be isometric towards the root (as after
 * ttn_sweep, or ttn_node_export of such a state).  Copies them to the device
 * (pinned host memory makes the copies asynchronous), rebuilds every
 * renormalized operator and puts the centre at the root.  QED_ENAN if an
 * entry is NaN or infinite (looked for on the device after the copies; the
 * state's tensors are then undefined until a load succeeds). */
int ttn_load_tensors(ttn_state *s, const double *const *bufs, const int64_t *sizes, int32_t n_nodes);
/* Kernels launched by the library in this process so far (all states). */
int qed_launch_count(int64_t *count);

/* y = H_eff x at the current centre (Methods step (i)), x and y in the
 * centre's block layout; host buffers (copied in and out).  Computed in the
 * state's precision: tensor-core TF32/BF16 products at bottom nodes of a
 * mixed-precision state, FP64 otherwise. */
int ttn_apply_heff(ttn_state *s, const double *x, double *y, int64_t n);
/* Same with device buffers on the state's stream (no host copies). */
int ttn_apply_heff_device(ttn_state *s, const double *x_device, double *y_device, int64_t n);

/* Checkpoint (no counterpart in the paper).  ttn_save moves the centre to the root (so the file holds a
 * tree isometric towards the root) and writes: the 8-byte tag "QEDTTN01",
 * the model parameters (Lx, Ly, Lz, boundary, Q as int32; t, m, ge2, cB, nu as
 * FP64), chi, precision (int32), seed (uint64), the node count (int32), the
 * node sizes (int64) and every node tensor (FP64, the ttn_node_export
 * layout), then an FNV-1a 64-bit hash of all preceding bytes; host byte
 * order.  ttn_load checks the tag, the hash and that the parameters equal
 * the model's (bitwise), creates a state on cuda_stream (ttn_create) and
 * loads the tensors (ttn_load_tensors); QED_EINVAL on any mismatch or I/O
 * error, *out NULL then.  Caller owns *out (ttn_destroy). */
int ttn_save(ttn_state *s, const char *path);
int ttn_load(const qed_model *m, const char *path, void *cuda_stream, ttn_state **out);

/* Differentiation of E(psi; couplings) = psi^T H_eff psi / psi^T psi.  The
 * paper updates tensors by the eigensolver only (Methods, steps (i)-(iii));
 * the gradient and the gradient step are additions, and dE/dcoupling rests
 * on Eq. (1) + Eq. (16) being linear in each coupling.
 *
 * y = H_eff^T x at the current centre with every product term transposed
 * (A^T (x) B^T (x) C^T on the three legs, monomial site operators through
 * inverse row maps): the hand-written adjoint of the H_eff contraction, FP64,
 * device buffers (n doubles, centre layout) on the state's stream.  H_eff
 * of Eq. (1) + Eq. (16) is real symmetric, so the result equals
 * ttn_apply_heff_device's (FP64 state) to rounding. */
int ttn_apply_heff_adjoint_device(ttn_state *s, const double *x_device, double *y_device, int64_t n);
/* Energy gradient with the centre moved to `node` (node < 0: current
 * centre).  psi_device: n doubles in the centre layout, or NULL for the
 * centre tensor.  Outputs: *energy; dE_dpsi_device (optional, n doubles) =
 * ((H + H^T) psi - 2 E psi) / psi^T psi, with H^T psi from the adjoint
 * product; dE_dcoupling[5] = dE/d(t, m, ge2, cB, nu).  E is linear in the
 * couplings, so each is the class expectation value divided by the coupling
 * (Hellmann-Feynman); NaN for a zero coupling (its terms are absent).  The
 * operator products are recomputed on every call (nothing is kept from an
 * earlier call).  All products FP64 whatever the state's precision. */
int ttn_energy_grad(ttn_state *s, int32_t node, const double *psi_device, int64_t n, double *energy,
                    double *dE_dpsi_device, double dE_dcoupling[5]);
/* Gradient node update on the centre tensor: psi <- (psi - eta dE/dpsi) /
 * |psi - eta dE/dpsi|, with the energies before and after. */
int ttn_gradient_step(ttn_state *s, double eta, double *e_before, double *e_after);

/* y = H_eff x at the current centre, allocating nothing: no cudaMalloc,
 * cudaFree or other allocating routine is called, on the device or the
 * host.  The paper has no counterpart; this exists for callers whose
 * device memory is owned by another allocator (a framework pool or an arena
 * fixed at start-up) and who cannot let a library allocate or free device
 * memory, which would also synchronise the device.
 *
 * Same product and FP64 grouped-GEMM kernel as ttn_apply_heff_device on an
 * FP64 state; x_device and y_device (n doubles, centre layout) are used in
 * place.  The kernel's work list lives in one file-scope device array of
 * 4 MiB that every GPU loading the library holds until the process exits.
 * The first call on a device looks up that array's device address once
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * The work list is written on the host into a static pageable buffer and
 * copied to the array with cudaMemcpyAsync on the state's stream; a copy
 * from pageable memory first waits for the work already queued on that
 * stream and returns once the host buffer has been read, so each call
 * blocks the calling thread until the stream's earlier work is done (the
 * kernel launch itself is asynchronous).
 * Every call rewrites the array, so kernels of calls that overlap on the GPU
 * race.  Two states have two different streams: calls on different
 * ttn_state objects (from one thread or several) can overlap, and the caller
 * must synchronise between them (for example cudaStreamSynchronize on the
 * first state's stream before calling on the second).  Calls on one state
 * are ordered on its stream.
 * The centre must be a bottom node whose row maps and environment operators
 * exist: any bottom node that ttn_move_center or a sweep moved the centre to
 * has them, because every operator update that leaves it builds them.  A
 * bottom node that is also the root (a two-site lattice) is never left by an
 * operator update; there one call of ttn_apply_heff_device at that centre
 * builds the row maps first.  Errors: QED_EUNSUPPORTED for another centre,
 * a missing row map (the message names it) or a work list larger than the
 * array, QED_EINVAL for a size mismatch. */
int ttn_apply_heff_device_noalloc(ttn_state *s, const double *x_device, double *y_device, int64_t n);

const char *qed_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* QEDTTN_H */
