"""Thin Python binding over libp4d.so (argument marshalling only)."""
import ctypes as C

import numpy as np
import torch

from . import _native as N


def default_params(**overrides):
    """p4d_params with the library defaults, overridden by keyword."""
    lib = N.load()
    p = N.Params()
    lib.p4d_params_default(C.byref(p))
    for k, v in overrides.items():
        if k in ("ocp_n", "ocp_p"):
            getattr(p, k)[0], getattr(p, k)[1] = float(v[0]), float(v[1])
        elif k == "order":
            for i in range(3):
                p.order[i] = int(v[i])
        else:
            setattr(p, k, v)
    return p


_PHYS_KEYS = ("F", "R", "T", "tplus", "brug", "De", "kappa", "sigma_n", "sigma_p", "k_n", "k_p", "cmax_n",
              "cmax_p", "alpha", "ocp_n", "ocp_p", "dt", "i_app", "diffpot_sign")


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _dev(t):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    return t


class P4DSolver:
    """One cell: mesh + parameters -> a libp4d handle.

    case: dict with "mesh" (arrays as produced by ``p4d_inputs``) and
    "params" (physical constants); solver options are keyword arguments
    (precision, combine, order, restart, maxit, mode, cheb_degree,
    coarse_max, cheb_ratio, rtol).
    """

    def __init__(self, case, device="cuda", stream=None, **opts):
        self.lib = N.load()
        m = case["mesh"]
        phys = {k: case["params"][k] for k in _PHYS_KEYS if k in case["params"]}
        self.params = default_params(**phys, **opts)
        self._keep = []

        def dp(a):
            a = np.ascontiguousarray(a, dtype=np.float64)
            self._keep.append(a)
            return a.ctypes.data_as(C.POINTER(C.c_double))

        def up(a):
            a = np.ascontiguousarray(a, dtype=np.uint8)
            self._keep.append(a)
            return a.ctypes.data_as(C.POINTER(C.c_uint8))

        mesh = N.Mesh(nx=int(m["nx"]), ny=int(m["ny"]), nz=int(m["nz"]), hx=dp(m["hx"]), hy=dp(m["hy"]),
                      hz=dp(m["hz"]), region=up(m["region"]), eps=dp(m["eps"]), eps_s=dp(m["eps_s"]),
                      Rs=dp(m["Rs"]), Ds=dp(m["Ds"]), gamma_p=up(m["gamma_p"]), gamma_n=up(m["gamma_n"]),
                      rgrid=dp(m["rgrid"]), nc=int(m["nc"]),
                      sigma_e=dp(m["sigma_e"]) if m.get("sigma_e") is not None else None,
                      Ds_e=dp(m["Ds_e"]) if m.get("Ds_e") is not None else None,
                      shell_sigma_t_p=float(m.get("shell_sigma_t_p", 0.0) or 0.0),
                      shell_sigma_t_n=float(m.get("shell_sigma_t_n", 0.0) or 0.0))
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = C.c_void_p()
        st = self.lib.p4d_setup(C.byref(mesh), C.byref(self.params), None, C.c_void_p(self.stream.cuda_stream),
                                C.byref(h))
        N.check(st, "p4d_setup")
        self.h = h
        self._nelem = int(m["nx"]) * int(m["ny"]) * int(m["nz"])
        nn, ne, nd, nc = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int32()
        N.check(self.lib.p4d_get_sizes(h, C.byref(nn), C.byref(ne), C.byref(nd), C.byref(nc)), "p4d_get_sizes")
        self.nn, self.NE, self.ndof, self.nc = nn.value, ne.value, nd.value, nc.value
        en = np.zeros(max(self.NE, 1), np.int32)
        N.check(self.lib.p4d_electrode_nodes(h, en.ctypes.data_as(C.POINTER(C.c_int32))), "p4d_electrode_nodes")
        self.enodes = en[: self.NE]

    # ----------------------------------------------------------------- state
    def state_tensors(self, st):
        """Device tensors of a generator state (c_s rows of electrode nodes)."""
        d = self.device
        f = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float64), device=d)
        return dict(phis=f(st["phis"]), phie=f(st["phie"]), ce=f(st["ce"]),
                    cs=f(np.asarray(st["cs_node"])[self.enodes]), ce_prev=f(st["ce_prev"]),
                    cs_prev=f(np.asarray(st["cs_prev_node"])[self.enodes]))

    def _state(self, s):
        for k in ("phis", "phie", "ce", "cs", "ce_prev", "cs_prev"):
            _dev(s[k])
        return N.State(phis=_ptr(s["phis"]), phie=_ptr(s["phie"]), ce=_ptr(s["ce"]), cs=_ptr(s["cs"]),
                       ce_prev=_ptr(s["ce_prev"]), cs_prev=_ptr(s["cs_prev"]))

    # ----------------------------------------------------------------- calls
    def residual(self, s, out=None):
        out = torch.empty(self.ndof, dtype=torch.float64, device=self.device) if out is None else _dev(out)
        N.check(self.lib.p4d_residual(self.h, C.byref(self._state(s)), _ptr(out)), "p4d_residual")
        return out

    def jacobian_update(self, s):
        N.check(self.lib.p4d_jacobian_update(self.h, C.byref(self._state(s))), "p4d_jacobian_update")

    def jvp(self, x, transpose=False, out=None):
        out = torch.empty_like(x) if out is None else out
        N.check(self.lib.p4d_jvp(self.h, _ptr(_dev(x)), _ptr(_dev(out)), int(transpose)), "p4d_jvp")
        return out

    def precond(self, r, transpose=False, out=None):
        out = torch.empty_like(r) if out is None else out
        N.check(self.lib.p4d_precond_apply(self.h, _ptr(_dev(r)), _ptr(_dev(out)), int(transpose)),
                "p4d_precond_apply")
        return out

    def set_options(self, **opts):
        for k, v in opts.items():
            if k == "order":
                for i in range(3):
                    self.params.order[i] = int(v[i])
            else:
                setattr(self.params, k, v)
        N.check(self.lib.p4d_set_params(self.h, C.byref(self.params)), "p4d_set_params")

    def solve(self, b, x=None, adjoint=False, check=True):
        """FGMRES solve of J x = b (adjoint: J^T x = b); returns (x, info dict)."""
        x = torch.zeros_like(b) if x is None else x
        info = N.Info()
        fn = self.lib.p4d_adjoint_solve if adjoint else self.lib.p4d_fgmres_solve
        st = fn(self.h, _ptr(_dev(b)), _ptr(_dev(x)), C.byref(info))
        if check and st not in (N.OK,):
            raise N.P4DError(st, "p4d_fgmres_solve")
        d = info.as_dict()
        d["status"] = st
        return x, d

    def newton(self, s, rtol=1e-10, maxit=20):
        """Newton solve of one backward-Euler step in place on s["phis"],
        s["phie"], s["ce"], s["cs"] (previous level s["ce_prev"], s["cs_prev"])."""
        it = C.c_int32()
        info = N.Info()
        st = self.lib.p4d_newton_solve(self.h, _ptr(_dev(s["phis"])), _ptr(_dev(s["phie"])), _ptr(_dev(s["ce"])),
                                       _ptr(_dev(s["cs"])), _ptr(_dev(s["ce_prev"])), _ptr(_dev(s["cs_prev"])),
                                       float(rtol), int(maxit), C.byref(it), C.byref(info))
        N.check(st, "p4d_newton_solve")
        return it.value, info.as_dict()

    def voltage_weights(self):
        q = torch.empty(self.ndof, dtype=torch.float64, device=self.device)
        N.check(self.lib.p4d_voltage_weights(self.h, _ptr(q)), "p4d_voltage_weights")
        return q

    def terminal_voltage(self, phis):
        """V = mean of phi_s over Gamma_p, as a one-element device tensor."""
        v = torch.empty(1, dtype=torch.float64, device=self.device)
        N.check(self.lib.p4d_terminal_voltage(self.h, _ptr(_dev(phis)), _ptr(v)), "p4d_terminal_voltage")
        return v

    def param_grad(self, s, lam, g_sigma, g_Ds, g_eps):
        N.check(self.lib.p4d_param_grad(self.h, C.byref(self._state(s)), _ptr(_dev(lam)), _ptr(_dev(g_sigma)),
                                        _ptr(_dev(g_Ds)), _ptr(_dev(g_eps))), "p4d_param_grad")

    def adjoint_prev(self, lam, out=None):
        out = torch.empty_like(lam) if out is None else out
        N.check(self.lib.p4d_adjoint_prev(self.h, _ptr(_dev(lam)), _ptr(_dev(out))), "p4d_adjoint_prev")
        return out

    def close(self):
        if getattr(self, "h", None):
            self.lib.p4d_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def halo_plan(nplanes, ghosts=1):
    """Halo messages of z slabs with nplanes[p] local node planes and `ghosts`
    ghost planes per interior side: [(src slab, first src plane, dst slab,
    first dst plane)], `ghosts` planes each (p4d_dd_halo_plan; host only)."""
    lib = N.load()
    n = len(nplanes)
    arr = (C.c_int32 * n)(*[int(v) for v in nplanes])
    m = lib.p4d_dd_halo_plan(n, arr, int(ghosts), None)
    if m < 0:
        raise ValueError("a slab owns no node plane, or fewer than the ghost planes")
    out = (C.c_int32 * max(4 * m, 1))()
    lib.p4d_dd_halo_plan(n, arr, int(ghosts), out)
    return [tuple(out[4 * i:4 * i + 4]) for i in range(m)]


class SlabSolver:
    """One cell cut into z slabs (``p4d_inputs.slab_cases``): one handle per
    slab, all on one stream, grouped by p4d_dd_create.  Vectors are lists of
    per-slab device tensors in each slab's full layout."""

    def __init__(self, slabs, device="cuda", stream=None, coarse=2, **opts):
        self.slabs = slabs
        dev = torch.device(device)
        stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self.parts = [P4DSolver(s["case"], device=dev, stream=stream, **opts) for s in slabs]
        self.lib = self.parts[0].lib
        n = len(self.parts)
        hs = (C.c_void_p * n)(*[p.h.value for p in self.parts])
        out = C.c_void_p()
        N.check(self.lib.p4d_dd_create(hs, n, int(slabs[0]["ghosts"]), C.byref(out)), "p4d_dd_create")
        self.dd = out
        self.set_coarse(coarse)

    def set_coarse(self, modes):
        """Coarse space: 0 none, 1 constants, 2 constants and linear in z (next update)."""
        N.check(self.lib.p4d_dd_set_coarse(self.dd, int(modes)), "p4d_dd_set_coarse")

    def _ptrs(self, ts):
        return (C.c_void_p * len(ts))(*[_dev(t).data_ptr() for t in ts])

    def state_tensors(self):
        return [p.state_tensors(s["case"]["state"]) for p, s in zip(self.parts, self.slabs)]

    def residual(self, states):
        return [p.residual(s) for p, s in zip(self.parts, states)]

    def jacobian_update(self, states):
        arr = (N.State * len(self.parts))(*[p._state(s) for p, s in zip(self.parts, states)])
        N.check(self.lib.p4d_dd_jacobian_update(self.dd, arr), "p4d_dd_jacobian_update")

    def jvp(self, xs):
        """J x on the owned rows (the ghost planes of each x[p] receive the owners' values)."""
        ys = [torch.empty_like(x) for x in xs]
        N.check(self.lib.p4d_dd_jvp(self.dd, self._ptrs(xs), self._ptrs(ys)), "p4d_dd_jvp")
        return ys

    def solve(self, bs, xs=None, check=True):
        xs = [torch.zeros_like(b) for b in bs] if xs is None else xs
        info = N.Info()
        st = self.lib.p4d_dd_fgmres_solve(self.dd, self._ptrs(bs), self._ptrs(xs), C.byref(info))
        if check and st != N.OK:
            raise N.P4DError(st, "p4d_dd_fgmres_solve")
        d = info.as_dict()
        d["status"] = st
        return xs, d

    def close(self):
        if getattr(self, "dd", None):
            self.lib.p4d_dd_destroy(self.dd)
            self.dd = None
        for p in getattr(self, "parts", []):
            p.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
