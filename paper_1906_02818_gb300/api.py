"""Python binding of the C ABI (include/mc.h): argument marshalling only.

PyTorch provides device memory and streams; every simulation step runs in the
library's CUDA kernels.  Model and configuration are plain keyword arguments:

  model:  kind="gbm", s0, sigma, corr=None, weights=None, r, loadings=None ([d, k] factor model)
          kind="heston", s0, v0, r, kappa, theta, xi, rho
  cfg:    steps, T, paths, seed=42, scheme="log_euler", precision="fp32",
          path_offset=0, ckpt_every=0, monitoring="discrete" | "bridge"
  payoff: dict(kind=<name in native.PAYOFF>, strike=K, barrier=H)
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import native
from .native import McModel, McPayoff, McResult, McSimCfg, check


class _Marshalled:
    """Keeps the numpy arrays alive while the C structs point at them."""

    def __init__(self, model: dict, cfg: dict, payoffs=None):
        kind = model.get("kind", "gbm")
        self.arrays = []
        m = McModel()
        m.kind = native.MODEL[kind]
        s0 = self._arr(np.atleast_1d(model["s0"]))
        m.d = s0.size
        self.model_d = m.d
        m.s0 = self._ptr(s0)
        if kind == "gbm":
            # the library reads d (sigma, weights), d x d (corr) and d x k
            # (loadings) doubles through these pointers: the sizes are checked here
            m.sigma = self._ptr(self._sized(model["sigma"], m.d, "sigma"))
            if model.get("corr") is not None:
                m.corr = self._ptr(self._sized(model["corr"], m.d * m.d, "corr (d x d)"))
            if model.get("weights") is not None:
                m.weights = self._ptr(self._sized(model["weights"], m.d, "weights"))
            if model.get("loadings") is not None:
                B = np.asarray(model["loadings"], dtype=np.float64)
                if (B.ndim == 2 and B.shape[0] != m.d) or B.ndim > 2 or B.size % m.d:
                    raise ValueError(f"loadings of shape {B.shape} are not [d, k] with d = {m.d}")
                B = self._arr(B.reshape(m.d, -1))
                m.n_factors = B.shape[1]
                m.loadings = self._ptr(B) if B.size else self._ptr(self._arr(np.zeros(1)))
        else:
            for k in ("v0", "kappa", "theta", "xi", "rho"):
                setattr(m, k, float(model[k]))
        m.r = float(model["r"])
        self.model = m
        c = McSimCfg()
        c.scheme = native.SCHEME[cfg.get("scheme", "log_euler")]
        c.steps = int(cfg["steps"])
        c.T = float(cfg["T"])
        c.paths = int(cfg["paths"])
        c.path_offset = int(cfg.get("path_offset", 0))
        c.seed = int(cfg.get("seed", 42))
        c.precision = native.PRECISION[cfg.get("precision", "fp32")]
        c.ckpt_every = int(cfg.get("ckpt_every", 0))
        c.monitoring = native.MONITORING[cfg.get("monitoring", "discrete")]
        self.cfg = c
        self.n_payoff = 0
        self.payoffs = None
        if payoffs is not None:
            n = len(payoffs)
            arr = (McPayoff * max(n, 1))()
            for i, p in enumerate(payoffs):
                arr[i].kind = native.PAYOFF[p["kind"]]
                arr[i].strike = float(p.get("strike", 0.0))
                arr[i].barrier = float(p.get("barrier", float("inf")))
            self.payoffs = arr
            self.n_payoff = n

    def _arr(self, a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        self.arrays.append(a)
        return a

    def _sized(self, a, n, what):
        a = self._arr(np.atleast_1d(a))
        if a.size != n:
            raise ValueError(f"{what} has {a.size} entries, {n} expected for d = {self.model_d}")
        return a

    @staticmethod
    def _ptr(a):
        return a.ctypes.data_as(native.c_double_p)


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _cuda_f32(x, what):
    """x as a contiguous CUDA float32 tensor: the library reads float32
    device memory through the pointer, so any other tensor is refused."""
    import torch
    if not (torch.is_tensor(x) and x.is_cuda and x.dtype == torch.float32):
        raise ValueError(f"{what} must be a CUDA float32 tensor")
    return x.contiguous()


def _rows(x, cols, what):
    """A CUDA float32 [n, cols] tensor."""
    x = _cuda_f32(x, what)
    if x.dim() != 2 or x.shape[1] != cols:
        raise ValueError(f"{what} must have shape [n, {cols}], not {tuple(x.shape)}")
    return x


def _count(x, n, what):
    """A CUDA float32 tensor of exactly n values."""
    x = _cuda_f32(x, what)
    if x.numel() != n:
        raise ValueError(f"{what} holds {x.numel()} values, {n} expected")
    return x


def _host_f32(a, n, what):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.size != n:
        raise ValueError(f"{what} holds {a.size} values, {n} expected")
    return a


def price(model: dict, cfg: dict, payoffs, stream=None):
    """Discounted prices and standard errors: list of (price, se)."""
    L = native.lib()
    mm = _Marshalled(model, cfg, payoffs)
    out = (McResult * mm.n_payoff)()
    check(L.mc_price(ctypes.byref(mm.model), ctypes.byref(mm.cfg), mm.payoffs, mm.n_payoff, out,
                     _stream_handle(stream)))
    return [(r.price, r.se) for r in out]


def price_mlmc(model: dict, cfg: dict, payoffs, paths_ref: int, stream=None):
    """Two-level precision estimator (mc_price_mlmc): cfg["precision"] is the
    coarse level's operand type on cfg["paths"] paths, paths_ref further
    paths carry the FP32 - reduced-precision correction.  Returns one dict
    per payoff: price, se, and (price, se) of coarse, correction, ref_level,
    coarse_level."""
    L = native.lib()
    mm = _Marshalled(model, cfg, payoffs)
    out = (native.McMlmcResult * mm.n_payoff)()
    check(L.mc_price_mlmc(ctypes.byref(mm.model), ctypes.byref(mm.cfg), mm.payoffs, mm.n_payoff, int(paths_ref), out,
                          _stream_handle(stream)))
    return [dict(price=r.price, se=r.se, coarse=(r.coarse.price, r.coarse.se),
                 correction=(r.correction.price, r.correction.se), ref_level=(r.ref_level.price, r.ref_level.se),
                 coarse_level=(r.coarse_level.price, r.coarse_level.se)) for r in out]


def price_qmc(model: dict, cfg: dict, payoffs, replications: int = 16, stream=None):
    """Randomised Sobol quasi-Monte Carlo (mc_price_qmc): cfg["paths"] points
    per replication.  Returns (list of (price, se), replication means
    [replications, n_payoff])."""
    L = native.lib()
    mm = _Marshalled(model, cfg, payoffs)
    out = (McResult * mm.n_payoff)()
    reps = np.zeros((replications, mm.n_payoff))
    check(L.mc_price_qmc(ctypes.byref(mm.model), ctypes.byref(mm.cfg), mm.payoffs, mm.n_payoff, int(replications),
                         out, reps.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _stream_handle(stream)))
    return [(r.price, r.se) for r in out], reps


def greeks(model: dict, cfg: dict, payoffs, stream=None):
    """Pathwise Greeks: (prices, greeks) with prices a list of (price, se) and
    greeks an array [n_payoff, G, 2] of (mean, se); G = 7 for Heston
    (S0, v0, r, kappa, theta, xi, rho), 2d + 1 for GBM with d assets
    (d/dS0_a for every asset, then d/dsigma_a, then d/dr)."""
    L = native.lib()
    mm = _Marshalled(model, cfg, payoffs)
    G = L.mc_greek_count(ctypes.byref(mm.model))
    pr = (McResult * mm.n_payoff)()
    gr = (McResult * (mm.n_payoff * G))()
    check(L.mc_greeks(ctypes.byref(mm.model), ctypes.byref(mm.cfg), mm.payoffs, mm.n_payoff, pr, gr,
                      _stream_handle(stream)))
    g = _results_np(gr, (mm.n_payoff, G, 2))
    return [(r.price, r.se) for r in pr], g


def _results_np(arr, shape):
    """A ctypes array of mc_result (two doubles each) as a float64 copy of
    the given shape, without a Python loop over the entries."""
    return np.frombuffer(arr, dtype=np.float64).reshape(shape).copy()


def corr_greeks(model: dict, cfg: dict, payoff: dict, stream=None):
    """Pathwise correlation sensitivities of one European basket call or put
    (mc_corr_greeks): ((price, se), dl [d, d, 2], drho [d, d, 2]) with
    dl[a, b] = (mean, se) of dP/dLrho[a][b] (b <= a) and drho[a, b] of
    dP/dcorr[a][b] (a != b, both entries moved)."""
    L = native.lib()
    mm = _Marshalled(model, cfg, [payoff])
    d = mm.model.d
    pr = McResult()
    dl = (McResult * (d * d))()
    dr = (McResult * (d * d))()
    check(L.mc_corr_greeks(ctypes.byref(mm.model), ctypes.byref(mm.cfg), mm.payoffs, ctypes.byref(pr), dl, dr,
                           _stream_handle(stream)))
    a = _results_np(dl, (d, d, 2))
    b = _results_np(dr, (d, d, 2))
    return (pr.price, pr.se), a, b


def simulate(model: dict, cfg: dict, save_every: int = 1, stream=None):
    """Simulated paths as a CUDA float32 tensor [steps/save_every + 1, D, paths]."""
    import torch
    L = native.lib()
    mm = _Marshalled(model, cfg)
    D = 2 if model.get("kind", "gbm") == "heston" else mm.model.d
    nsave = mm.cfg.steps // save_every + 1 if save_every > 0 else 0
    out = torch.empty((nsave, D, mm.cfg.paths), dtype=torch.float32, device="cuda")
    check(L.mc_simulate(ctypes.byref(mm.model), ctypes.byref(mm.cfg), int(save_every),
                        ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)))
    return out


def moments(results, paths: int) -> np.ndarray:
    """(N mean, N mean(f^2), N) per payoff [n, 3] of a run's (price, se)
    list over `paths` paths (mc_moments)."""
    n = len(results)
    res = (McResult * n)(*[McResult(float(p), float(se)) for p, se in results])
    out = np.empty((n, 3), dtype=np.float64)
    check(native.lib().mc_moments(res, n, int(paths), out.ctypes.data_as(native.c_double_p)))
    return out


def combine(mom) -> list:
    """(price, se) per payoff from moments summed over runs (mc_combine)."""
    mom = np.ascontiguousarray(mom, dtype=np.float64).reshape(-1, 3)
    out = (McResult * mom.shape[0])()
    check(native.lib().mc_combine(mom.ctypes.data_as(native.c_double_p), mom.shape[0], out))
    return [(r.price, r.se) for r in out]


def tail(dev_pnl, alpha: float = 0.99, stream=None) -> dict:
    """VaR / CVaR of the losses -pnl of a CUDA float64 vector (mc_tail)."""
    pnl = dev_pnl.contiguous()
    if not pnl.is_cuda or pnl.dtype.itemsize != 8 or pnl.dim() != 1:
        raise ValueError("dev_pnl must be a 1-D CUDA float64 tensor")
    res = native.McRiskResult()
    check(native.lib().mc_tail(ctypes.c_void_p(pnl.data_ptr()), pnl.numel(), float(alpha), ctypes.byref(res),
                               _stream_handle(stream)))
    return dict(var=res.var, cvar=res.cvar, n_tail=res.n_tail)


def philox_words(seed: int, stream_index: int, q0: int, blocks: int, stream=None):
    """Philox4x32-10 blocks q0 .. q0 + blocks - 1 of a stream (mc_philox_words)
    as a CUDA int32 tensor [blocks, 4] holding the uint32 words' bits."""
    import torch
    out = torch.empty((max(blocks, 1), 4), dtype=torch.int32, device="cuda")
    check(native.lib().mc_philox_words(int(seed), int(stream_index), int(q0), int(blocks),
                                       ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)))
    return out[:blocks]


def normals(seed: int, stream_index: int, j0: int, count: int, stream=None):
    """Normals j0 .. j0 + count - 1 of a stream (mc_normals), CUDA float32 [count]."""
    import torch
    out = torch.empty(max(count, 1), dtype=torch.float32, device="cuda")
    check(native.lib().mc_normals(int(seed), int(stream_index), int(j0), int(count),
                                  ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)))
    return out[:count]


class Plan:
    """A set-up computation (mc_plan_create) executable asynchronously."""

    def __init__(self, model: dict, cfg: dict, payoffs, stream=None):
        self._lib = native.lib()
        mm = _Marshalled(model, cfg, payoffs)
        self.n_payoff = mm.n_payoff
        h = ctypes.c_void_p()
        check(self._lib.mc_plan_create(ctypes.byref(mm.model), ctypes.byref(mm.cfg), mm.payoffs,
                                       mm.n_payoff, ctypes.byref(h), _stream_handle(stream)))
        self._h = h

    def execute(self, out=None, stream=None):
        """Launch on `stream`; returns the CUDA float64 tensor [n_payoff, 2] of
        (price, se) that the launch will fill."""
        import torch
        if out is None:
            out = torch.empty((self.n_payoff, 2), dtype=torch.float64, device="cuda")
        check(self._lib.mc_plan_execute(self._h, ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)))
        return out

    @property
    def launches(self) -> int:
        return self._lib.mc_plan_launches(self._h)

    def close(self):
        if self._h:
            self._lib.mc_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Mlp:
    """The surrogate network (mc_mlp_*): parameters on the device, forward in
    FP32 or BF16, loss/gradient and native Adam training."""

    def __init__(self, n_in: int, width: int, hidden: int, init):
        self._lib = native.lib()
        init = np.ascontiguousarray(init, dtype=np.float32)
        h = ctypes.c_void_p()
        check(self._lib.mc_mlp_create(n_in, width, hidden, init.ctypes.data_as(ctypes.c_void_p), ctypes.byref(h)))
        self._h = h
        self.n_in = n_in
        self.count = self._lib.mc_mlp_param_count(h)
        if self.count != init.size:
            self.close()
            raise ValueError(f"init has {init.size} values, the network {self.count}")

    @property
    def handle(self):
        return self._h

    def params(self) -> np.ndarray:
        out = np.empty(self.count, dtype=np.float32)
        check(self._lib.mc_mlp_get_params(self._h, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def set_params(self, p):
        p = _host_f32(p, self.count, "params")
        check(self._lib.mc_mlp_set_params(self._h, p.ctypes.data_as(ctypes.c_void_p)))

    def set_train_mode(self, mode: str):
        """Arithmetic of loss_grad / train: "fp32" (FP32 SIMT products) or
        "tf32x3" (width -> width products on the tensor cores, three-pass TF32)."""
        code = {"fp32": native.MC_MLP_TRAIN_FP32, "tf32x3": native.MC_MLP_TRAIN_TF32X3}[mode]
        check(self._lib.mc_mlp_set_train_mode(self._h, code))

    def forward(self, x, precision="fp32", stream=None):
        import torch
        x = _rows(x, self.n_in, "x")
        y = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
        check(self._lib.mc_mlp_forward(self._h, ctypes.c_void_p(x.data_ptr()), x.shape[0], ctypes.c_void_p(y.data_ptr()),
                                       native.PRECISION[precision], _stream_handle(stream)))
        return y

    def loss_grad(self, x, t, stream=None):
        x = _rows(x, self.n_in, "x")
        t = _count(t, x.shape[0], "t")
        g = np.empty(self.count, dtype=np.float32)
        loss = ctypes.c_double()
        check(self._lib.mc_mlp_loss_grad(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                         x.shape[0], ctypes.byref(loss), g.ctypes.data_as(ctypes.c_void_p),
                                         _stream_handle(stream)))
        return loss.value, g

    def train(self, x, t, epochs, batch, lr, stream=None):
        x = _rows(x, self.n_in, "x")
        t = _count(t, x.shape[0], "t")
        loss = ctypes.c_double()
        check(self._lib.mc_mlp_train(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                     x.shape[0], epochs, batch, ctypes.c_float(lr), ctypes.byref(loss),
                                     _stream_handle(stream)))
        return loss.value

    def apply_grad(self, g, lr, stream=None):
        """One Adam step with the given packed gradient (host array)."""
        g = _host_f32(g, self.count, "g")
        check(self._lib.mc_mlp_apply_grad(self._h, g.ctypes.data_as(ctypes.c_void_p), ctypes.c_float(lr),
                                          _stream_handle(stream)))

    @staticmethod
    def _dloss(dirs, scales, weights):
        if len(dirs) > 4 or not (len(dirs) == len(scales) == len(weights)):
            raise ValueError("up to 4 directions, with one scale and one weight each")
        d = native.McMlpDloss()
        d.n_dir = len(dirs)
        for k, (j, sc, wt) in enumerate(zip(dirs, scales, weights)):
            d.dir[k], d.scale[k], d.weight[k] = int(j), float(sc), float(wt)
        return d

    def loss_grad_d(self, x, t, g, dirs, scales, weights, stream=None):
        """Loss with derivative labels (mc_mlp_loss_grad_d): (loss parts
        [1 + K], packed gradient); g a CUDA float32 [n, K] tensor (NaN: no
        label)."""
        x = _rows(x, self.n_in, "x")
        t = _count(t, x.shape[0], "t")
        d = self._dloss(dirs, scales, weights)
        gp = ctypes.c_void_p(_count(g, x.shape[0] * d.n_dir, "g").data_ptr()) if d.n_dir else None
        parts = (ctypes.c_double * (1 + d.n_dir))()
        grad = np.empty(self.count, dtype=np.float32)
        check(self._lib.mc_mlp_loss_grad_d(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(t.data_ptr()), gp,
                                           x.shape[0], ctypes.byref(d), parts, grad.ctypes.data_as(ctypes.c_void_p),
                                           _stream_handle(stream)))
        return list(parts), grad

    def train_d(self, x, t, g, dirs, scales, weights, epochs, batch, lr, stream=None):
        """Mini-batch Adam on the derivative-label loss (mc_mlp_train_d)."""
        x = _rows(x, self.n_in, "x")
        t = _count(t, x.shape[0], "t")
        d = self._dloss(dirs, scales, weights)
        gp = ctypes.c_void_p(_count(g, x.shape[0] * d.n_dir, "g").data_ptr()) if d.n_dir else None
        loss = ctypes.c_double()
        check(self._lib.mc_mlp_train_d(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(t.data_ptr()), gp,
                                       x.shape[0], ctypes.byref(d), epochs, batch, ctypes.c_float(lr),
                                       ctypes.byref(loss), _stream_handle(stream)))
        return loss.value

    def loss_grad_sums(self, x, t, stream=None):
        """CUDA float32 [count + 1]: the gradient of the batch's summed
        squared error and that sum (mc_mlp_loss_grad_sums, asynchronous)."""
        import torch
        x = _rows(x, self.n_in, "x")
        t = _count(t, x.shape[0], "t")
        out = torch.empty(self.count + 1, dtype=torch.float32, device=x.device)
        check(self._lib.mc_mlp_loss_grad_sums(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                              x.shape[0], ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)))
        return out

    def apply_grad_sums(self, g, scale, lr, stream=None):
        """One Adam step with gradient scale * g[:count] (g a CUDA float32
        tensor; mc_mlp_apply_grad_sums, asynchronous)."""
        g = _cuda_f32(g, "g")
        if g.numel() < self.count:
            raise ValueError(f"g holds {g.numel()} values, at least {self.count} expected")
        check(self._lib.mc_mlp_apply_grad_sums(self._h, ctypes.c_void_p(g.data_ptr()), ctypes.c_float(scale),
                                               ctypes.c_float(lr), _stream_handle(stream)))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mc_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


PORTFOLIO_KIND = {0: 0, 1: 1, 4: 4}  # call, put, up-and-out call (mc_payoff_kind codes)


def surrogate_labels(points, paths, steps_per_year=252, seed=42, stream=None, with_inputs=False):
    """Monte Carlo training labels V_call / K at CUDA float32 points [n, 5]
    (S/K, sigma, tau, r, K/H); with_inputs=True also returns the network
    inputs of the points."""
    import torch
    pts = _rows(points, 5, "points")
    out = torch.empty(pts.shape[0], dtype=torch.float32, device=pts.device)
    inp = torch.empty_like(pts) if with_inputs else None
    check(native.lib().mc_surrogate_labels(pts.shape[0], ctypes.c_void_p(pts.data_ptr()), paths, steps_per_year, seed,
                                           ctypes.c_void_p(out.data_ptr()),
                                           ctypes.c_void_p(inp.data_ptr()) if with_inputs else None,
                                           _stream_handle(stream)))
    return (out, inp) if with_inputs else out


def surrogate_label_greeks(points, paths, steps_per_year=252, seed=42, stream=None, with_inputs=False):
    """Labels and their pathwise Greeks (mc_surrogate_label_greeks): (labels
    [n], dlabels [n, 2] = (d/d(S/K), d/d sigma), NaN rows for barrier points
    [, inputs])."""
    import torch
    pts = _rows(points, 5, "points")
    out = torch.empty(pts.shape[0], dtype=torch.float32, device=pts.device)
    dl = torch.empty((pts.shape[0], 2), dtype=torch.float32, device=pts.device)
    inp = torch.empty_like(pts) if with_inputs else None
    check(native.lib().mc_surrogate_label_greeks(pts.shape[0], ctypes.c_void_p(pts.data_ptr()), paths, steps_per_year,
                                                 seed, ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(dl.data_ptr()),
                                                 ctypes.c_void_p(inp.data_ptr()) if with_inputs else None,
                                                 _stream_handle(stream)))
    return (out, dl, inp) if with_inputs else (out, dl)


def risk(portfolio: dict, alpha=0.99, n_scen=1 << 16, method="nested", inner_paths=1 << 12, base_paths=1 << 16,
         seed=42, surrogate=None, surrogate_precision="fp32", want_pnl=False, scen_offset=0, stream=None):
    """VaR / CVaR of the portfolio (see mc_risk) over scenarios
    [scen_offset, scen_offset + n_scen); returns a dict."""
    L = native.lib()
    keep = []

    # the library reads n_under (s0, sigma), n_under^2 (corr) and n_opt (the
    # option arrays) values through these pointers: the sizes are checked here
    def sized(x, n, what, dtype):
        a = np.ascontiguousarray(np.atleast_1d(x), dtype=dtype)
        if a.size != n:
            raise ValueError(f"portfolio {what} has {a.size} entries, {n} expected")
        keep.append(a)
        return a

    def dp(x, n, what):
        return sized(x, n, what, np.float64).ctypes.data_as(native.c_double_p)

    def ip(x, n, what):
        return sized(x, n, what, np.int32).ctypes.data_as(ctypes.POINTER(ctypes.c_int32))

    pf = native.McPortfolio()
    d = pf.n_under = len(np.atleast_1d(portfolio["s0"]))
    pf.s0, pf.sigma = dp(portfolio["s0"], d, "s0"), dp(portfolio["sigma"], d, "sigma")
    pf.corr = dp(portfolio["corr"], d * d, "corr") if portfolio.get("corr") is not None else None
    pf.r, pf.mu = float(portfolio["r"]), float(portfolio["mu"])
    no = pf.n_opt = len(np.atleast_1d(portfolio["strike"]))
    pf.under = ip(portfolio["under"], no, "under")
    kinds = [int(k) for k in np.atleast_1d(portfolio["kind"])]
    if any(k not in PORTFOLIO_KIND for k in kinds):
        raise ValueError("portfolio option kinds: 0 call, 1 put, 4 up-and-out call")
    pf.kind = ip([PORTFOLIO_KIND[k] for k in kinds], no, "kind")
    pf.strike, pf.barrier = dp(portfolio["strike"], no, "strike"), dp(portfolio["barrier"], no, "barrier")
    pf.maturity, pf.position = dp(portfolio["maturity"], no, "maturity"), dp(portfolio["position"], no, "position")
    cf = native.McRiskCfg()
    cf.alpha, cf.horizon, cf.n_scen = alpha, float(portfolio["horizon"]), int(n_scen)
    cf.steps_per_year = int(portfolio.get("steps_per_year", 252))
    cf.method = native.RISK_METHOD[method]
    cf.inner_paths, cf.base_paths, cf.seed = int(inner_paths), int(base_paths), int(seed)
    cf.surrogate = surrogate.handle if surrogate is not None else None
    cf.surrogate_precision = native.PRECISION[surrogate_precision]
    cf.scen_offset = int(scen_offset)
    res = native.McRiskResult()
    pnl = np.empty(int(n_scen)) if want_pnl else None
    check(L.mc_risk(ctypes.byref(pf), ctypes.byref(cf), ctypes.byref(res),
                    pnl.ctypes.data_as(ctypes.c_void_p) if want_pnl else None, _stream_handle(stream)))
    out = dict(var=res.var, cvar=res.cvar, base_value=res.base_value, n_tail=res.n_tail)
    if want_pnl:
        out["pnl"] = pnl
    return out
