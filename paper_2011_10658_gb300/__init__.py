"""GB300-native TTN hot path for (3+1)D lattice QED (arXiv:2011.10658).

Thin Python layer over the C ABI of include/qedttn.h.  Every computation
runs in libqedttn.so (host model code and sm_103a kernels); this module only
marshals arguments.
"""
import ctypes

import numpy as np

from . import _lib
from ._lib import QedDrive, QedDriveRecord, QedDriveState, QedError, QedParams, SweepStats, check, lib

PREC = {"fp64": 0, "tf32": 1, "bf16": 2, "tf32x3": 3}
OP = {"I": 0, "M": 1, "MD": 2, "C": 3, "P": 4, "N": 5, "E2": 6, "PC": 8}
MEAS = {"probs": 0, "phi": 1, "nx": 2, "qx": 3, "k": 4, "elink": 5, "scalars": 6, "sigma": 7}
CLASSES = ("t", "m", "ge2", "cB", "nu")   # scalar couplings; terms of class 5 are the chemical potentials


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def launch_count():
    """Kernels launched by libqedttn in this process."""
    n = ctypes.c_int64()
    check(lib().qed_launch_count(ctypes.byref(n)))
    return n.value


def basis(parity):
    """Dressed-site basis table [267, 9] (phi, k1..k6, sign, q)."""
    out = np.zeros((267, 9), dtype=np.int8)
    n = ctypes.c_int32()
    check(lib().qed_basis(parity, _ptr(out, ctypes.c_int8), ctypes.byref(n)))
    return out[: n.value]


def local_op(parity, kind, j1=0, j2=0):
    """Monomial site operator: (src[267] int16, val[267] float64)."""
    src = np.zeros(267, dtype=np.int16)
    val = np.zeros(267, dtype=np.float64)
    k = OP[kind] if isinstance(kind, str) else int(kind)
    check(lib().qed_local_op(parity, k, j1, j2, _ptr(src, ctypes.c_int16), _ptr(val, ctypes.c_double)))
    return src, val


def batch_sweep(states, n=1, tol=1e-12, max_krylov=64, allow_noconv=False):
    """n sweeps of several independent TTN states together (ttn_batch_sweep);
    one stats dict per state."""
    k = len(states)
    handles = (ctypes.c_void_p * k)(*[st._h.value for st in states])
    stats = (SweepStats * k)()
    check(lib().ttn_batch_sweep(handles, k, n, tol, max_krylov, stats), allow=(-4,) if allow_noconv else ())
    return [dict(energy=st.energy, matvecs=st.matvecs, matvecs_mixed=st.matvecs_mixed,
                 node_updates=st.node_updates, not_converged=st.not_converged,
                 max_rel_residual=st.max_rel_residual, seconds=st.seconds) for st in stats]


DRIVE_DEFAULTS = dict(nu_start=0.5, nu_step=0.5, quad_coef=0.25, nu_max=10.0, tol_start=1e-4, tol_factor=0.1,
                      tol_final=1e-10, conv_rel=1e-8, rise_rel=1e-9, min_final_sweeps=2, max_sweeps=40,
                      max_krylov=64)


def drive_settings(**kw):
    """qed_drive with DRIVE_DEFAULTS overridden by kw."""
    unknown = set(kw) - set(DRIVE_DEFAULTS)
    if unknown:
        raise TypeError(f"unknown drive settings {sorted(unknown)}")
    return QedDrive(**dict(DRIVE_DEFAULTS, **kw))


def drive_start(d):
    """qed_drive_start: schedule state of sweep 0."""
    st = QedDriveState()
    check(lib().qed_drive_start(ctypes.byref(d), ctypes.byref(st)))
    return st


def drive_next(d, st, energy):
    """qed_drive_next: advance st past a sweep that ended at `energy`."""
    check(lib().qed_drive_next(ctypes.byref(d), ctypes.byref(st), float(energy)))
    return st


class Model:
    """Lattice, term list and tree (qed_model_create)."""

    def __init__(self, Lx, Ly, Lz, t=1.0, m=1.0, ge2=1.0, cB=0.5, nu=10.0, Q=0, boundary=0, mu=None):
        """boundary: 0 open, 1 periodic; mu: chemical potential per site
        (qed_model_set_site_potential), None for none."""
        self.params = QedParams(Lx, Ly, Lz, boundary, t, m, ge2, cB, nu, Q)
        h = ctypes.c_void_p()
        check(lib().qed_model_create(ctypes.byref(self.params), ctypes.byref(h)))
        self._h = h
        if mu is not None:
            self.set_site_potential(mu)

    def set_site_potential(self, mu):
        mu = np.ascontiguousarray(mu, dtype=np.float64)
        check(lib().qed_model_set_site_potential(self._h, _ptr(mu, ctypes.c_double), mu.size))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().qed_model_destroy(h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def info(self):
        ns, nt, nn = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        c = ctypes.c_double()
        check(lib().qed_model_info(self._h, ctypes.byref(ns), ctypes.byref(nt), ctypes.byref(nn), ctypes.byref(c)))
        return dict(n_sites=ns.value, n_terms=nt.value, n_nodes=nn.value, constant=c.value)

    def terms(self):
        n = ctypes.c_int64()
        check(lib().qed_model_terms(self._h, None, None, None, None, 0, ctypes.byref(n)))
        cnt = n.value
        coef = np.zeros(cnt)
        cls = np.zeros(cnt, dtype=np.int32)
        nops = np.zeros(cnt, dtype=np.int32)
        ops = np.zeros((cnt, 4, 4), dtype=np.int32)
        check(lib().qed_model_terms(self._h, _ptr(coef, ctypes.c_double), _ptr(cls, ctypes.c_int32),
                                    _ptr(nops, ctypes.c_int32), _ptr(ops, ctypes.c_int32), cnt, ctypes.byref(n)))
        return coef, cls, nops, ops

    def tree(self):
        n = ctypes.c_int64()
        check(lib().qed_model_tree(self._h, None, 0, ctypes.byref(n)))
        out = np.zeros((n.value, 7), dtype=np.int32)
        check(lib().qed_model_tree(self._h, _ptr(out, ctypes.c_int32), n.value, ctypes.byref(n)))
        return out

    def sweep_order(self):
        """Node ids in the order one sweep updates them."""
        n = ctypes.c_int64()
        check(lib().qed_model_sweep_order(self._h, None, 0, ctypes.byref(n)))
        out = np.zeros(n.value, dtype=np.int32)
        check(lib().qed_model_sweep_order(self._h, _ptr(out, ctypes.c_int32), n.value, ctypes.byref(n)))
        return out

    def sectors(self, chi):
        """List over nodes of {q: dim} for the bond above each node."""
        n = ctypes.c_int64()
        check(lib().qed_model_sectors(self._h, chi, None, 0, ctypes.byref(n)))
        out = np.zeros((n.value, 3), dtype=np.int32)
        check(lib().qed_model_sectors(self._h, chi, _ptr(out, ctypes.c_int32), n.value, ctypes.byref(n)))
        nn = self.info()["n_nodes"]
        bonds = [dict() for _ in range(nn)]
        for node, q, d in out:
            bonds[int(node)][int(q)] = int(d)
        return bonds


class TTN:
    """Device-resident TTN state (ttn_create).  ``stream``: an integer
    cudaStream_t (e.g. torch.cuda.current_stream().cuda_stream) or None."""

    def __init__(self, model, chi, seed=0, precision="fp64", stream=None):
        self.model = model
        h = ctypes.c_void_p()
        check(lib().ttn_create(model.handle, chi, seed, PREC[precision], ctypes.c_void_p(stream or 0),
                               ctypes.byref(h)))
        self._h = h
        self.chi = chi

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().ttn_destroy(h)
            self._h = None

    def __del__(self):
        self.close()

    def sweep(self, n=1, tol=1e-12, max_krylov=64, allow_noconv=False):
        st = SweepStats()
        check(lib().ttn_sweep(self._h, n, tol, max_krylov, ctypes.byref(st)), allow=(-4,) if allow_noconv else ())
        return dict(energy=st.energy, matvecs=st.matvecs, matvecs_mixed=st.matvecs_mixed, node_updates=st.node_updates,
                    not_converged=st.not_converged, max_rel_residual=st.max_rel_residual, seconds=st.seconds)

    def set_couplings(self, t, m, ge2, cB, nu):
        """ttn_set_couplings: new couplings, operators rebuilt, centre at the root."""
        c = np.array([t, m, ge2, cB, nu], dtype=np.float64)
        check(lib().ttn_set_couplings(self._h, _ptr(c, ctypes.c_double)))

    def drive(self, allow_noconv=False, **settings):
        """ttn_drive with drive_settings(**settings); (records, converged)."""
        d = drive_settings(**settings)
        cap = d.max_sweeps
        log = (QedDriveRecord * cap)()
        n = ctypes.c_int32()
        rc = check(lib().ttn_drive(self._h, ctypes.byref(d), log, cap, ctypes.byref(n)),
                   allow=(-4,) if allow_noconv else ())
        recs = [{f: getattr(log[i], f) for f, _ in QedDriveRecord._fields_} for i in range(min(n.value, cap))]
        return recs, rc == 0

    def optimize_node(self, node, tol=1e-12, max_krylov=64):
        e = ctypes.c_double()
        check(lib().ttn_optimize_node(self._h, node, tol, max_krylov, ctypes.byref(e)))
        return e.value

    def set_precision(self, precision):
        check(lib().ttn_set_precision(self._h, PREC[precision]))

    def set_mixed_tol(self, tol):
        check(lib().ttn_set_mixed_tol(self._h, tol))

    def set_wait_limit(self, polls):
        check(lib().ttn_set_wait_limit(self._h, int(polls)))

    def last_update(self):
        a, b, r = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
        th, rm = ctypes.c_double(), ctypes.c_double()
        check(lib().ttn_last_update(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(r), ctypes.byref(th),
                                    ctypes.byref(rm)))
        return dict(iters_fp64=a.value, iters_mixed=b.value, rel_residual=r.value, ritz_mixed=th.value,
                    rel_residual_mixed=rm.value)

    def set_profiling(self, on=True):
        check(lib().ttn_set_profiling(self._h, 1 if on else 0))

    def reset_timing(self):
        check(lib().ttn_reset_timing(self._h))

    def kernel_timing(self, kernel_class):
        ms, n, fa, fe, ba = (ctypes.c_double(), ctypes.c_int64(), ctypes.c_double(), ctypes.c_double(),
                             ctypes.c_double())
        k = {"tc_heff": 0, "heff_simt_bottom": 1, "heff_simt_upper": 2, "heff_upper": 2, "move": 3,
             "lanczos": 4, "move_qr": 5, "move_ops": 6, "move_ops_upper": 6,
             "move_ops_bottom": 7}.get(kernel_class, kernel_class)
        check(lib().ttn_kernel_timing(self._h, k, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(fa),
                                      ctypes.byref(fe), ctypes.byref(ba)))
        return dict(ms=ms.value, launches=n.value, flops_alg=fa.value, flops_exec=fe.value, bytes_alg=ba.value)

    def move_center(self, node):
        check(lib().ttn_move_center(self._h, node))

    def info(self):
        c, nn, mx = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
        check(lib().ttn_info(self._h, ctypes.byref(c), ctypes.byref(nn), ctypes.byref(mx)))
        return dict(center=c.value, n_nodes=nn.value, max_node_size=mx.value)

    def node_size(self, node):
        n = ctypes.c_int64()
        check(lib().ttn_node_size(self._h, node, ctypes.byref(n)))
        return n.value

    def energy(self):
        """(E_total, E_without_penalty, {class: <H_class>})."""
        et, ew = ctypes.c_double(), ctypes.c_double()
        parts = np.zeros(5)
        check(lib().ttn_energy(self._h, ctypes.byref(et), ctypes.byref(ew), _ptr(parts, ctypes.c_double)))
        return et.value, ew.value, dict(zip(CLASSES, parts.tolist()))

    def measure(self, kind):
        k = MEAS[kind]
        n = ctypes.c_int64()
        check(lib().ttn_measure(self._h, k, None, 0, ctypes.byref(n)))
        out = np.zeros(n.value)
        check(lib().ttn_measure(self._h, k, _ptr(out, ctypes.c_double), n.value, ctypes.byref(n)))
        return out

    def node_export(self, node):
        n = self.node_size(node)
        out = np.zeros(n)
        nn = ctypes.c_int64()
        check(lib().ttn_node_export(self._h, node, _ptr(out, ctypes.c_double), n, ctypes.byref(nn)))
        return out

    def node_import(self, node, data):
        data = np.ascontiguousarray(data, dtype=np.float64)
        check(lib().ttn_node_import(self._h, node, _ptr(data, ctypes.c_double), data.size))

    def load_tensors(self, arrays):
        """arrays: one float64 buffer per node (numpy arrays or integer host
        pointers with sizes as (ptr, n) pairs)."""
        n = len(arrays)
        ptrs = (ctypes.POINTER(ctypes.c_double) * n)()
        sizes = np.zeros(n, dtype=np.int64)
        keep = []
        for i, a in enumerate(arrays):
            if isinstance(a, tuple):
                ptrs[i] = ctypes.cast(ctypes.c_void_p(a[0]), ctypes.POINTER(ctypes.c_double))
                sizes[i] = a[1]
            else:
                a = np.ascontiguousarray(a, dtype=np.float64)
                keep.append(a)
                ptrs[i] = _ptr(a, ctypes.c_double)
                sizes[i] = a.size
        check(lib().ttn_load_tensors(self._h, ptrs, _ptr(sizes, ctypes.c_int64), n))

    def apply_heff(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.zeros_like(x)
        check(lib().ttn_apply_heff(self._h, _ptr(x, ctypes.c_double), _ptr(y, ctypes.c_double), x.size))
        return y

    def apply_heff_device(self, x_ptr, y_ptr, n):
        check(lib().ttn_apply_heff_device(self._h, ctypes.c_void_p(x_ptr), ctypes.c_void_p(y_ptr), n))

    def save(self, path):
        """Checkpoint (centre moved to the root first); see ttn_save."""
        check(lib().ttn_save(self._h, str(path).encode()))

    @classmethod
    def load(cls, model, path, stream=None):
        """State read from a ttn_save file for the same model."""
        h = ctypes.c_void_p()
        check(lib().ttn_load(model.handle, str(path).encode(), ctypes.c_void_p(stream or 0), ctypes.byref(h)))
        obj = cls.__new__(cls)
        obj.model = model
        obj._h = h
        obj.chi = None
        return obj

    def apply_heff_adjoint_device(self, x_ptr, y_ptr, n):
        """y = H_eff^T x (transposed terms, FP64) on device buffers."""
        check(lib().ttn_apply_heff_adjoint_device(self._h, ctypes.c_void_p(x_ptr), ctypes.c_void_p(y_ptr), n))

    def energy_grad_device(self, node=-1, psi_ptr=None, grad_ptr=None, n=0):
        """(E, {class: dE/dcoupling}) with the centre moved to ``node``, for the
        device vector at psi_ptr (n doubles) or the centre tensor; dE/dpsi is
        written to grad_ptr when given."""
        e = ctypes.c_double()
        dc = np.zeros(5)
        check(lib().ttn_energy_grad(self._h, node, ctypes.c_void_p(psi_ptr or 0), n, ctypes.byref(e),
                                    ctypes.c_void_p(grad_ptr or 0), _ptr(dc, ctypes.c_double)))
        return e.value, dict(zip(CLASSES, dc.tolist()))

    def gradient_step(self, eta):
        """psi <- normalize(psi - eta dE/dpsi) on the centre tensor; (E before, E after)."""
        e0, e1 = ctypes.c_double(), ctypes.c_double()
        check(lib().ttn_gradient_step(self._h, eta, ctypes.byref(e0), ctypes.byref(e1)))
        return e0.value, e1.value

    def apply_heff_device_noalloc(self, x_ptr, y_ptr, n):
        """Same product as apply_heff_device in FP64 at a bottom-node centre,
        with no memory allocated by the call (see include/qedttn.h)."""
        check(lib().ttn_apply_heff_device_noalloc(self._h, ctypes.c_void_p(x_ptr), ctypes.c_void_p(y_ptr), n))
