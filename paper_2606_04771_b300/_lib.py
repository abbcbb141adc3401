"""ctypes binding of the engine's C ABI (include/tdvp.h).

Argument marshalling only: every step of the method runs inside the CUDA
library.  Importing this module loads ``libtdvp.so`` and raises if it is
missing; there is no Python or CPU implementation behind these calls.
"""
from __future__ import annotations

import ctypes as C
import os
import struct

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtdvp.so")

SYM = {"u1u1": 0, "u1su2": 1, "su2": 1}
PREC = {"fp64": 0, "3xtf32": 1, "bf16x4": 2}
ERRORS = {0: "ok", -1: "EINVAL", -2: "ESTATE", -3: "ENOMEM", -4: "ENUMERIC", -5: "EINTERNAL", -6: "ECUDA",
          -7: "ETIMEOUT", -8: "ECANCELED", -9: "EIO"}
MODE = {"two": 0, "one": 1, "adaptive": 2}


class TdvpError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("krylov_max", C.c_int), ("krylov_tol", C.c_double),
                ("timeout_ms", C.c_int), ("cuda_stream", C.c_void_p), ("device", C.c_int),
                ("trunc_degeneracy", C.c_double), ("merge_launches", C.c_int)]


class RequestC(C.Structure):
    _fields_ = [("L", C.c_int), ("J", C.c_double), ("U", C.c_double), ("symmetry", C.c_int),
                ("precision", C.c_int), ("mode", C.c_int), ("dt", C.c_double), ("t_final", C.c_double),
                ("chi_max", C.c_longlong), ("eps", C.c_double), ("occupations", C.c_void_p)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is not built; run paper_2606_04771_b300/build.py")
        L = C.CDLL(LIB_PATH)
        P = C.POINTER
        vp = C.c_void_p
        sig = {
            "tdvp_opts_default": (None, [P(Opts)]),
            "tdvp_create": (C.c_int, [C.c_int, C.c_double, C.c_double, C.c_int, P(Opts), P(vp)]),
            "tdvp_step": (C.c_int, [vp, C.c_double, C.c_longlong, C.c_double]),
            "tdvp_step_mode": (C.c_int, [vp, C.c_double, C.c_longlong, C.c_double, C.c_int, P(C.c_int)]),
            "tdvp_create_random": (C.c_int, [C.c_int, C.c_double, C.c_double, C.c_int, C.c_longlong, C.c_ulonglong,
                                             C.c_int, P(Opts), P(vp)]),
            "tdvp_create_product": (C.c_int, [C.c_int, C.c_double, C.c_double, C.c_int, vp, P(Opts), P(vp)]),
            "tdvp_bond_update": (C.c_int, [vp, C.c_int, C.c_int, C.c_double, C.c_longlong, C.c_double, vp]),
            "tdvp_measure_center": (C.c_int, [vp, vp, vp, vp, vp]),
            "tdvp_measure": (C.c_int, [vp, vp, vp, vp, vp, vp]),
            "tdvp_bond_dims": (C.c_int, [vp, vp, vp]),
            "tdvp_stats": (C.c_int, [vp, vp, C.c_int]),
            "tdvp_bond_create": (C.c_int, [C.c_int, C.c_double, C.c_double, C.c_int, vp, C.c_int, vp, P(Opts),
                                           P(vp)]),
            "tdvp_block_count": (C.c_int, [vp, C.c_int, P(C.c_longlong), P(C.c_longlong)]),
            "tdvp_block_list": (C.c_int, [vp, C.c_int, vp, vp, vp]),
            "tdvp_set_tensor": (C.c_int, [vp, C.c_int, vp, C.c_longlong, C.c_int]),
            "tdvp_heff_apply": (C.c_int, [vp, C.c_int, vp, vp, C.c_int]),
            "tdvp_heff_flops": (C.c_int, [vp, P(C.c_longlong)]),
            "tdvp_krylov_expm": (C.c_int, [vp, C.c_int, vp, vp, C.c_double, C.c_int, P(C.c_int), P(C.c_int)]),
            "tdvp_heff_profile": (C.c_int, [vp, C.c_int, vp, vp, vp]),
            "tdvp_svd": (C.c_int, [C.c_int, C.c_int, vp, vp, vp, vp, C.c_int, vp]),
            "tdvp_svd_noalloc": (C.c_int, [C.c_int, C.c_int, vp, vp, vp, vp, vp]),
            "tdvp_truncate": (C.c_int, [C.c_int, vp, vp, vp, C.c_double, C.c_longlong, C.c_double, vp, vp, vp]),
            "tdvp_heff_groups": (C.c_int, [vp, P(C.c_int), vp, vp]),
            "tdvp_partition": (C.c_int, [C.c_int, vp, C.c_int, vp, vp]),
            "tdvp_heff_apply_owned": (C.c_int, [vp, C.c_int, vp, C.c_int, vp, vp, C.c_int]),
            "tdvp_launch_count": (C.c_int, [P(C.c_longlong)]),
            "tdvp_merge_count": (C.c_int, [P(C.c_longlong), P(C.c_longlong)]),
            "tdvp_selftest_wait": (C.c_int, [C.c_uint, vp]),
            "tdvp_destroy": (C.c_int, [vp]),
            "tdvp_save": (C.c_int, [vp, C.c_char_p, C.c_double]),
            "tdvp_load": (C.c_int, [C.c_char_p, P(Opts), P(vp), P(C.c_double)]),
            "tdvp_server_create": (C.c_int, [C.c_double, C.c_int, P(Opts), P(vp)]),
            "tdvp_server_footprint": (C.c_int, [P(RequestC), C.c_int, P(C.c_double)]),
            "tdvp_server_submit": (C.c_int, [vp, P(RequestC), P(C.c_longlong)]),
            "tdvp_server_poll": (C.c_int, [vp, C.c_longlong, P(C.c_int)]),
            "tdvp_server_wait": (C.c_int, [vp, C.c_longlong, C.c_int, P(C.c_int)]),
            "tdvp_server_result": (C.c_int, [vp, C.c_longlong, vp, vp, vp, vp, vp, C.c_int]),
            "tdvp_server_cancel": (C.c_int, [vp, C.c_longlong]),
            "tdvp_server_pause": (C.c_int, [vp, C.c_int]),
            "tdvp_server_stats": (C.c_int, [vp, vp, C.c_int]),
            "tdvp_server_destroy": (C.c_int, [vp]),
            "tdvp_strerror": (C.c_char_p, [C.c_int]),
            "tdvp_last_error": (C.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(rc):
    if rc != 0:
        raise TdvpError(rc, lib().tdvp_last_error().decode())


def make_opts(precision="fp64", krylov_max=20, krylov_tol=1e-12, stream=None, device=-1, trunc_degeneracy=None,
              merge_launches=False):
    o = Opts()
    lib().tdvp_opts_default(C.byref(o))
    o.merge_launches = 1 if merge_launches else 0
    if trunc_degeneracy is not None:
        o.trunc_degeneracy = float(trunc_degeneracy)
    o.precision = PREC[precision] if isinstance(precision, str) else int(precision)
    o.krylov_max = krylov_max
    o.krylov_tol = krylov_tol
    o.cuda_stream = stream
    o.device = device
    return o


def _ptr(x):
    """(pointer, on_device) for a numpy complex128 array or a torch tensor."""
    if isinstance(x, np.ndarray):
        assert x.dtype == np.complex128 and x.flags["C_CONTIGUOUS"]
        return x.ctypes.data, 0
    # torch tensor (complex128, contiguous); device pointer when on CUDA
    assert x.is_contiguous()
    return x.data_ptr(), 1 if x.is_cuda else 0


def svd(a, stream=None):
    """Thin SVD of a complex128 matrix through tdvp_svd: returns (u, s, vh).

    a is a numpy array (host path) or a CUDA torch tensor (device path)."""
    p, q = a.shape
    r = min(p, q)
    if isinstance(a, np.ndarray):
        a = np.ascontiguousarray(a, dtype=np.complex128)
        u = np.empty((p, r), np.complex128)
        vh = np.empty((r, q), np.complex128)
        s = np.empty(r)
        check(lib().tdvp_svd(p, q, a.ctypes.data, s.ctypes.data, u.ctypes.data, vh.ctypes.data, 0, stream))
        return u, s, vh
    import torch

    u = torch.empty((p, r), dtype=torch.complex128, device=a.device)
    vh = torch.empty((r, q), dtype=torch.complex128, device=a.device)
    s = torch.empty(r, dtype=torch.float64, device=a.device)
    check(lib().tdvp_svd(p, q, a.data_ptr(), s.data_ptr(), u.data_ptr(), vh.data_ptr(), 1, stream))
    return u, s, vh


def truncate(values, mults, eps, chi_max, degeneracy=0.0, stream=None):
    """The truncation's multiplet selection through tdvp_truncate.

    values: one descending 1-D array of reduced singular values per sector (sv^2 is
    the weight of a whole multiplet); mults: 2S+1 per sector.  Returns (kept per
    sector, stats) with stats = (total weight, discarded weight, 1/sqrt(kept
    weight), K, states kept, 1.0 when the chi cap set K)."""
    nsec = len(values)
    r = np.array([len(v) for v in values], dtype=np.int32)
    m = np.ascontiguousarray(mults, dtype=np.int32)
    sv = np.ascontiguousarray(np.concatenate([np.asarray(v, dtype=np.float64) for v in values]))
    kept = np.zeros(nsec, dtype=np.int32)
    stats = np.zeros(6)
    check(lib().tdvp_truncate(nsec, r.ctypes.data, m.ctypes.data, sv.ctypes.data, float(eps), int(chi_max),
                              float(degeneracy), kept.ctypes.data, stats.ctypes.data, stream))
    return kept, stats


def merge_count():
    """(launches that carried more than one context's GEMM work, task lists they carried)."""
    a, b = C.c_longlong(), C.c_longlong()
    check(lib().tdvp_merge_count(C.byref(a), C.byref(b)))
    return a.value, b.value


def launch_count():
    """Kernel launches this library has enqueued in the process so far."""
    n = C.c_longlong()
    check(lib().tdvp_launch_count(C.byref(n)))
    return n.value


class _Ctx:
    def __init__(self):
        self.h = C.c_void_p()

    def close(self):
        if self.h:
            check(lib().tdvp_destroy(self.h))
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def blocks(self, which):
        nb, ne = C.c_longlong(), C.c_longlong()
        check(lib().tdvp_block_count(self.h, which, C.byref(nb), C.byref(ne)))
        keys = np.zeros((nb.value, 5), dtype=np.int32)
        dims = np.zeros((nb.value, 2), dtype=np.int32)
        offs = np.zeros(nb.value, dtype=np.int64)
        check(lib().tdvp_block_list(self.h, which, keys.ctypes.data, dims.ctypes.data, offs.ctypes.data))
        return keys, dims, offs, ne.value

    def heff_apply(self, psi, out=None):
        if out is None:
            out = np.empty_like(psi) if isinstance(psi, np.ndarray) else psi.new_empty(psi.shape)
        pi, di = _ptr(psi)
        po, do = _ptr(out)
        assert di == do
        check(lib().tdvp_heff_apply(self.h, 0, pi, po, di))
        return out

    def heff_groups(self):
        """The output groups of the last GEMM stage: (flops per group, group of each
        output block) as int64 / int32 arrays."""
        ng = C.c_int()
        check(lib().tdvp_heff_groups(self.h, C.byref(ng), None, None))
        flops = np.zeros(ng.value, dtype=np.int64)
        nb = C.c_longlong()
        ne = C.c_longlong()
        check(lib().tdvp_block_count(self.h, 0, C.byref(nb), C.byref(ne)))
        bg = np.zeros(nb.value, dtype=np.int32)
        check(lib().tdvp_heff_groups(self.h, C.byref(ng), flops.ctypes.data, bg.ctypes.data))
        return flops, bg

    def heff_apply_owned(self, owner, rank, psi, out):
        """out = H_eff psi on the output groups g with owner[g] == rank (device tensors;
        the other blocks of out are left as they were)."""
        ow = np.ascontiguousarray(owner, dtype=np.int32)
        pi, di = _ptr(psi)
        po, do = _ptr(out)
        assert di == 1 and do == 1, "device tensors"
        check(lib().tdvp_heff_apply_owned(self.h, 0, ow.ctypes.data, int(rank), pi, po, 1))
        return out

    def krylov_expm(self, psi, out=None, tau=0.025):
        """out = exp(-i tau H_eff) psi; returns out.  Records the Krylov dimension used."""
        if out is None:
            out = np.empty_like(psi) if isinstance(psi, np.ndarray) else psi.new_empty(psi.shape)
        pi, di = _ptr(psi)
        po, do = _ptr(out)
        assert di == do
        k, nl = C.c_int(), C.c_int()
        check(lib().tdvp_krylov_expm(self.h, 0, pi, po, tau, di, C.byref(k), C.byref(nl)))
        self._kdim, self._launches = k.value, nl.value
        return out

    def last_krylov_dim(self):
        return self._kdim

    def launches_per_step(self):
        return self._launches

    def heff_flops(self):
        f = C.c_longlong()
        check(lib().tdvp_heff_flops(self.h, C.byref(f)))
        return f.value


def vacancy_occupations(L):
    """The benchmark's second initial state: the Neel pattern (up on even sites, down on
    odd sites) with the centre site L // 2 empty."""
    occ = [1 if i % 2 == 0 else 2 for i in range(L)]
    occ[L // 2] = 0
    return occ


class Chain(_Ctx):
    """An L-site chain in the Neel state (or, with random_chi, a synthetic random
    right-canonical state of that bond dimension), evolved with tdvp_step."""

    def __init__(self, L, J=1.0, U=4.0, symmetry="su2", random_chi=None, seed=1, center=0, occupations=None,
                 **opts):
        """occupations: per site 0 (empty), 1 (up), 2 (down), 3 (both) -- a product initial
        state instead of the Neel state (e.g. the central-vacancy state)."""
        super().__init__()
        self.L = L
        self.sym = symmetry
        o = make_opts(**opts)
        if occupations is not None:
            occ = np.ascontiguousarray(np.array(occupations, dtype=np.int32))
            assert occ.shape == (L,)
            check(lib().tdvp_create_product(L, J, U, SYM[symmetry], occ.ctypes.data, C.byref(o), C.byref(self.h)))
        elif random_chi is None:
            check(lib().tdvp_create(L, J, U, SYM[symmetry], C.byref(o), C.byref(self.h)))
        else:
            check(lib().tdvp_create_random(L, J, U, SYM[symmetry], int(random_chi), int(seed), int(center),
                                           C.byref(o), C.byref(self.h)))

    def save(self, path, t=0.0):
        """Checkpoint the chain (bond tables, site tensors, centre, adaptive state) and t."""
        check(lib().tdvp_save(self.h, os.fsencode(path), float(t)))

    @classmethod
    def load(cls, path, **opts):
        """A chain resumed from a checkpoint; returns (chain, t).  opts as for Chain
        (precision, krylov_max, krylov_tol, stream, device)."""
        ch = cls.__new__(cls)
        _Ctx.__init__(ch)
        o = make_opts(**opts)
        t = C.c_double()
        check(lib().tdvp_load(os.fsencode(path), C.byref(o), C.byref(ch.h), C.byref(t)))
        with open(path, "rb") as f:  # header: magic, int32 version, L, su2, ...
            _, _, L, su2 = struct.unpack("<8s3i", f.read(20))
        ch.L, ch.sym = L, ("su2" if su2 else "u1u1")
        return ch, t.value

    def step(self, dt, chi_max, eps, mode="two"):
        """One time step; mode "two" (two-site), "one" (one-site, bond dimensions
        fixed) or "adaptive" (two-site until the chi cap binds, then one-site).
        Returns the integrator used ("two" or "one")."""
        m = MODE[mode]
        used = C.c_int()
        check(lib().tdvp_step_mode(self.h, dt, int(chi_max), eps, m, C.byref(used)))
        return "one" if used.value == 1 else "two"

    def measure(self, entropy=True, energy=True):
        L = self.L
        n, sz, docc = np.zeros(L), np.zeros(L), np.zeros(L)
        ent = np.zeros(max(L - 1, 1))
        e = np.zeros(1)
        check(lib().tdvp_measure(self.h, n.ctypes.data, sz.ctypes.data, docc.ctypes.data,
                                 ent.ctypes.data if entropy else None, e.ctypes.data if energy else None))
        out = {"n": n, "sz": sz, "docc": docc, "n_up": 0.5 * n + sz, "n_dn": 0.5 * n - sz}
        if entropy:
            out["s_ent"] = ent[: L - 1]
        if energy:
            out["energy"] = float(e[0])
        return out

    def bond_update(self, bond, direction, dt, chi_max, eps):
        """One two-site update at (bond, bond+1); returns the new bond's entropy."""
        s = np.zeros(1)
        check(lib().tdvp_bond_update(self.h, bond, direction, dt, int(chi_max), eps, s.ctypes.data))
        return float(s[0])

    def measure_center(self):
        site = C.c_int()
        v = np.zeros(3)
        check(lib().tdvp_measure_center(self.h, C.byref(site), v[0:].ctypes.data, v[1:].ctypes.data,
                                        v[2:].ctypes.data))
        return site.value, {"n": v[0], "sz": v[1], "docc": v[2]}

    def bond_dims(self):
        chi = np.zeros(self.L + 1, dtype=np.int64)
        red = np.zeros(self.L + 1, dtype=np.int64)
        check(lib().tdvp_bond_dims(self.h, chi.ctypes.data, red.ctypes.data))
        return chi, red

    def stats(self):
        v = np.zeros(38)
        check(lib().tdvp_stats(self.h, v.ctypes.data, 38))
        keys = ["seconds", "heff_flops", "env_flops", "matvecs", "max_krylov", "max_discarded", "chi_max_seen",
                "t_theta", "t_plan", "t_krylov2", "t_split", "t_env", "t_krylov1", "steps", "splits", "sweeps64",
                "sweeps32", "one_site_steps", "device_bytes", "device_bytes_peak", "jacobi32_ms", "jacobi32_flops",
                "jacobi64_ms", "jacobi64_flops", "split_pmax", "split_qmax", "split_work", "split_work_small",
                "jacobi_calls", "jacobi_resident_calls", "jacobi_cluster_calls", "env_ms", "env_bytes", "gram_ms",
                "gram_flops", "gram_steps", "gram_fallbacks", "jacobi_ring_calls"]
        return dict(zip(keys, v.tolist()))


class BondProblem(_Ctx):
    """Two-site effective-Hamiltonian problem between two given bond sector tables."""

    def __init__(self, left, right, J=1.0, U=4.0, symmetry="su2", **opts):
        super().__init__()
        o = make_opts(**opts)
        lt = np.ascontiguousarray(np.array(left, dtype=np.int32).reshape(-1, 3))
        rt = np.ascontiguousarray(np.array(right, dtype=np.int32).reshape(-1, 3))
        check(lib().tdvp_bond_create(SYM[symmetry], J, U, lt.shape[0], lt.ctypes.data, rt.shape[0],
                                     rt.ctypes.data, C.byref(o), C.byref(self.h)))

    def set_env(self, which, data):
        p, dev = _ptr(data)
        n = data.size if isinstance(data, np.ndarray) else data.numel()
        check(lib().tdvp_set_tensor(self.h, which, p, n, dev))
