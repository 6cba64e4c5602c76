"""Thin Python layer over the fdcore C-ABI: handles, device buffers and streams.

Every computation runs in the library's kernels; this module only prepares
arguments (torch supplies device memory and streams) and owns handles.
"""
import ctypes
import hashlib
import math
import os

import numpy as np
import torch

from . import _lib as L
from . import fdgraph

_TAPE_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "tapes")
_JIT_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "jit")


def _stream_ptr(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def ueg_params(order, rs, T_over_TF, lam_over_kF, kext_over_kF, kc_over_kF=6.0):
    """fd_params of one instance (Rydberg units, eps = k^2 - mu, V = 8 pi/(q^2 + Lambda))."""
    kF = (9.0 * math.pi / 4.0) ** (1.0 / 3.0) / rs
    EF = kF * kF
    p = L.fd_params()
    p.k_ext = kext_over_kF * kF
    p.k_F = kF
    p.mu = EF
    p.beta = 1.0 / (T_over_TF * EF)
    p.Lambda = (lam_over_kF * kF) ** 2
    p.k_cut = kc_over_kF * kF
    p.order = order
    return p


DEFAULT_SCHEDULE = dict(budget=128, bundle=8, window=64)


def tape_bytes(order, roots, budget=None, bundle=None, window=None):
    """Compiled tape for (order, roots, schedule), cached on disk by compiler source hash."""
    sch = dict(DEFAULT_SCHEDULE)
    for k, v in (("budget", budget), ("bundle", bundle), ("window", window)):
        if v is not None:
            sch[k] = v
    src = open(fdgraph.__file__, "rb").read()
    key = hashlib.sha1(src + repr((order, list(roots), sorted(sch.items()))).encode()).hexdigest()[:16]
    path = os.path.join(_TAPE_DIR, "tape_o%d_%s.bin" % (order, key))
    if os.path.exists(path):
        return open(path, "rb").read()
    data = fdgraph.compile_graph(order, roots, **sch).to_bytes()
    os.makedirs(_TAPE_DIR, exist_ok=True)
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "wb") as f:
        f.write(data)
    os.replace(tmp, path)
    return data


def jit_options(threads=128, min_blocks=2, max_modules=None, root_units=True, sync_every=0, leaf_calls=False, spt=1,
                unit_cap=6000, pair=False, sv_smem=False, cross_roots=False, leaf_cache=0, lc_global=False):
    if max_modules is None:
        max_modules = max(1, min(32, os.cpu_count() or 1))
    return L.fd_jit_options(threads, min_blocks, max_modules, 1 if root_units else 0, sync_every,
                            1 if leaf_calls else 0, spt, unit_cap, 1 if pair else 0, 1 if sv_smem else 0,
                            1 if cross_roots else 0, int(leaf_cache), 1 if lc_global else 0)


def jit_source(tape, module=0, **options):
    """Generated source of one module of the specialised kernel (no device needed):
    (text, module count).  Options as Graph.jit."""
    opt = jit_options(**options)
    n = ctypes.c_int64()
    nm = ctypes.c_int32()
    L.check(L.lib().fd_jit_emit(tape, len(tape), ctypes.byref(opt), module, None, 0, ctypes.byref(n),
                                ctypes.byref(nm)))
    buf = ctypes.create_string_buffer(n.value + 1)
    L.check(L.lib().fd_jit_emit(tape, len(tape), ctypes.byref(opt), module, buf, n.value + 1, ctypes.byref(n),
                                ctypes.byref(nm)))
    return buf.value.decode(), nm.value


class Graph:
    """A compiled self-energy graph loaded on the current device."""

    def __init__(self, order, roots=None, with_dk=False, tape=None, budget=None, bundle=None, window=None):
        self.order = order
        self.roots = list(roots) if roots is not None else fdgraph.graph_roots(order, with_dk)
        data = tape if tape is not None else tape_bytes(order, self.roots, budget, bundle, window)
        self.tape = data
        self._buf = ctypes.create_string_buffer(data, len(data))
        h = ctypes.c_void_p()
        L.check(L.lib().fd_graph_load(self._buf, len(data), ctypes.byref(h)))
        self.handle = h
        nr, dim, ns = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        ni = ctypes.c_int64()
        L.check(L.lib().fd_graph_info(h, ctypes.byref(nr), ctypes.byref(dim), ctypes.byref(ni), ctypes.byref(ns)))
        self.n_roots, self.dim, self.n_instr, self.n_slots = nr.value, dim.value, ni.value, ns.value

    def set_launch(self, threads=0, samples_per_thread=0):
        L.check(L.lib().fd_graph_set_launch(self.handle, threads, samples_per_thread))

    def jit(self, cache=True, **options):
        """Compile the specialised straight-line kernel (cached under _build/jit)
        and evaluate this graph with it from now on.  Options (fd_jit_options):
        threads, min_blocks, max_modules, root_units, sync_every, leaf_calls,
        spt, unit_cap, pair, sv_smem, cross_roots, leaf_cache, lc_global."""
        opt = jit_options(**options)
        cdir = _JIT_DIR if cache else None
        if cdir:
            os.makedirs(cdir, exist_ok=True)
        L.check(L.lib().fd_graph_jit(self.handle, ctypes.byref(opt), cdir.encode() if cdir else None))
        return self.jit_info()

    def jit_enable(self, on=True):
        L.check(L.lib().fd_graph_jit_enable(self.handle, 1 if on else 0))

    def jit_info(self):
        info = (ctypes.c_int32 * 6)()
        secs = ctypes.c_double()
        L.check(L.lib().fd_graph_jit_info(self.handle, info, ctypes.byref(secs)))
        return dict(threads=info[0], min_blocks=info[1], regs=info[2], local_bytes=info[3], modules=info[4],
                    enabled=bool(info[5]), compile_s=secs.value)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and L._lib is not None:
            L._lib.fd_graph_free(h)
            self.handle = None


class Vegas:
    """VEGAS map of one instance (FP64 edges on the device)."""

    def __init__(self, dim, n_bins=1024):
        h = ctypes.c_void_p()
        L.check(L.lib().fd_vegas_create(dim, n_bins, ctypes.byref(h)))
        self.handle, self.dim, self.n_bins = h, dim, n_bins

    def set_edges(self, edges):
        e = np.ascontiguousarray(edges, dtype=np.float64)
        assert e.shape == (self.dim, self.n_bins + 1)
        L.check(L.lib().fd_vegas_set_edges(self.handle, e.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))

    def edges(self):
        e = np.empty((self.dim, self.n_bins + 1))
        L.check(L.lib().fd_vegas_get_edges(self.handle, e.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return e

    def hist(self):
        h = np.empty((self.dim, self.n_bins))
        L.check(L.lib().fd_vegas_get_hist(self.handle, h.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return h

    def set_hist(self, hist):
        h = np.ascontiguousarray(hist, dtype=np.float64)
        assert h.shape == (self.dim, self.n_bins)
        L.check(L.lib().fd_vegas_set_hist(self.handle, h.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))

    def clear(self, stream=None):
        L.check(L.lib().fd_vegas_clear_hist(self.handle, _stream_ptr(stream)))

    def update(self, alpha=0.5, stream=None):
        L.check(L.lib().fd_vegas_update(self.handle, alpha, _stream_ptr(stream)))

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and L._lib is not None:
            L._lib.fd_vegas_free(h)
            self.handle = None


def map_samples(vegas, seed, it, inst, n, dim, stream=None):
    x = torch.empty((dim, n), dtype=torch.float32, device="cuda")
    w = torch.empty((n,), dtype=torch.float32, device="cuda")
    L.check(L.lib().fd_map_samples(vegas.handle if vegas else None, seed, it, inst, n, dim, _ptr(x), _ptr(w),
                                   _stream_ptr(stream)))
    return x, w


class EvalPlan:
    """Launch description of one batched fd_integrand_eval call (reusable buffers)."""

    def __init__(self, graphs, params, graph_of_inst, n_per_inst, maps=None, per_sample=False):
        self.graphs = list(graphs)
        self.n_inst = len(params)
        self.n_per_inst = int(n_per_inst)
        self.r_max = max(g.n_roots for g in self.graphs)
        self.dim_max = max(g.dim for g in self.graphs)
        self._g = (ctypes.c_void_p * len(self.graphs))(*[g.handle for g in self.graphs])
        self._p = (L.fd_params * self.n_inst)(*params)
        self._gi = (ctypes.c_int32 * self.n_inst)(*graph_of_inst)
        self.maps = maps
        self._m = None
        if maps is not None:
            self._m = (ctypes.c_void_p * self.n_inst)(*[m.handle if m is not None else None for m in maps])
        cnt = L.lib().fd_partials_count(self.n_inst, self.r_max, self.n_per_inst)
        self.partials = torch.zeros(cnt, dtype=torch.float64, device="cuda")
        self.stats = torch.zeros((self.n_inst, self.r_max, 2, 2), dtype=torch.float64, device="cuda")
        self.per_sample = None
        if per_sample:
            self.per_sample = torch.zeros((self.n_inst, self.r_max, 2, self.n_per_inst), dtype=torch.float32,
                                          device="cuda")

    def run(self, seed, it, points=None, point_w=None, stream=None):
        L.check(L.lib().fd_integrand_eval(self._g, len(self.graphs), self._p, self._gi, self.n_inst, self._m,
                                          _ptr(points), _ptr(point_w), seed, it, self.n_per_inst,
                                          _ptr(self.partials), _ptr(self.per_sample), _stream_ptr(stream)))
        L.check(L.lib().fd_accumulate(_ptr(self.partials), self.n_inst, self.r_max, self.n_per_inst,
                                      _ptr(self.stats), _stream_ptr(stream)))
        return self.stats

    def run_target(self, seed, it, abs_f, points=None, point_w=None, stream=None):
        """Evaluate and write the training target (sum over value roots of
        |Re| + |Im|, weighted) per sample into abs_f [n_inst][n] (device FP32)."""
        L.check(L.lib().fd_integrand_eval_target(self._g, len(self.graphs), self._p, self._gi, self.n_inst, self._m,
                                                 _ptr(points), _ptr(point_w), seed, it, self.n_per_inst,
                                                 _ptr(self.partials), _ptr(abs_f), _stream_ptr(stream)))
        L.check(L.lib().fd_accumulate(_ptr(self.partials), self.n_inst, self.r_max, self.n_per_inst,
                                      _ptr(self.stats), _stream_ptr(stream)))
        return self.stats


class Flow:
    """Affine coupling flow with BF16 tensor-core kernels (FP32 master weights)."""

    def __init__(self, dim, n_layers=8, hidden=128, seed=0):
        h = ctypes.c_void_p()
        L.check(L.lib().fd_flow_create(dim, n_layers, hidden, seed, ctypes.byref(h)))
        self.handle, self.dim, self.n_layers, self.hidden = h, dim, n_layers, hidden
        self.n_params = L.lib().fd_flow_param_count(h)

    def set_params(self, blob):
        b = np.ascontiguousarray(blob, dtype=np.float32)
        assert b.size == self.n_params
        L.check(L.lib().fd_flow_set_params(self.handle, b.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), b.size))

    def params(self):
        b = np.empty(self.n_params, dtype=np.float32)
        L.check(L.lib().fd_flow_get_params(self.handle, b.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), b.size))
        return b

    def sample(self, seed, it, inst, n, stream=None):
        x = torch.empty((self.dim, n), dtype=torch.float32, device="cuda")
        w = torch.empty((n,), dtype=torch.float32, device="cuda")
        L.check(L.lib().fd_flow_sample(self.handle, seed, it, inst, n, _ptr(x), _ptr(w), _stream_ptr(stream)))
        return x, w

    def draw(self, seed, it, inst, n, stream=None):
        """Proposals: (x [dim][n], w = 1/q(x) [n]) (the flow's own sample stream)."""
        return self.sample(seed, it, inst, n, stream)

    def set_tensor_path(self, path):
        """Sampling / density on tcgen05, warp-specialised (2, default), tcgen05
        with tile pairs (1) or mma.sync (0)."""
        L.check(L.lib().fd_flow_set_tensor_path(self.handle, path))

    def sample_defensive(self, seed, it, inst, n, alpha, stream=None):
        """Mixture (1 - a) q_flow + a uniform: (x, w = 1/q_mix, a actually used)."""
        x = torch.empty((self.dim, n), dtype=torch.float32, device="cuda")
        w = torch.empty((n,), dtype=torch.float32, device="cuda")
        a = ctypes.c_double()
        L.check(L.lib().fd_flow_sample_defensive(self.handle, seed, it, inst, n, alpha, _ptr(x), _ptr(w),
                                                 ctypes.byref(a), _stream_ptr(stream)))
        return x, w, a.value

    def log_density(self, x, stream=None):
        n = x.shape[1]
        lq = torch.empty((n,), dtype=torch.float32, device="cuda")
        L.check(L.lib().fd_flow_log_density(self.handle, _ptr(x), n, _ptr(lq), _stream_ptr(stream)))
        return lq

    def grad(self, x, w, stream=None):
        n = x.shape[1]
        loss = torch.empty((1,), dtype=torch.float32, device="cuda")
        g = torch.empty((self.n_params,), dtype=torch.float32, device="cuda")
        L.check(L.lib().fd_flow_grad(self.handle, _ptr(x), _ptr(w), n, _ptr(loss), _ptr(g), _stream_ptr(stream)))
        return loss, g

    def train(self, x, w, steps, lr, stream=None):
        out = np.empty(steps, dtype=np.float32)
        L.check(L.lib().fd_flow_train(self.handle, _ptr(x), _ptr(w), x.shape[1], steps, lr,
                                      out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), _stream_ptr(stream)))
        return out

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and L._lib is not None:
            L._lib.fd_flow_free(h)
            self.handle = None


class SplineFlow:
    """Neural spline flow (App. A): rational-quadratic coupling layers on the
    unit hypercube; sampling, density and the training loss's gradient on the
    device (fd_nsf_*)."""

    def __init__(self, dim, n_layers=8):
        h = ctypes.c_void_p()
        L.check(L.lib().fd_nsf_create(dim, n_layers, ctypes.byref(h)))
        self.handle, self.dim, self.n_layers = h, dim, n_layers
        self.n_params = L.lib().fd_nsf_param_count(h)

    def set_params(self, blob):
        b = np.ascontiguousarray(blob, dtype=np.float32)
        assert b.size == self.n_params
        L.check(L.lib().fd_nsf_set_params(self.handle, b.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), b.size))

    def params(self):
        out = np.empty(self.n_params, dtype=np.float32)
        L.check(L.lib().fd_nsf_get_params(self.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                          out.size))
        return out

    def set_tensor_path(self, path):
        """Conditioner of the sampling / density passes on BF16 tensor cores (1,
        default) or FP32 CUDA cores (0)."""
        L.check(L.lib().fd_nsf_set_tensor_path(self.handle, path))

    def forward(self, z, stream=None):
        n = z.shape[1]
        x = torch.empty((self.dim, n), dtype=torch.float32, device="cuda")
        lq = torch.empty((n,), dtype=torch.float32, device="cuda")
        assert z.dtype == torch.float32 and z.is_contiguous() and z.shape[0] == self.dim
        L.check(L.lib().fd_nsf_forward(self.handle, _ptr(z), n, _ptr(x), _ptr(lq), _stream_ptr(stream)))
        return x, lq

    def sample(self, seed, it, inst, n, stream=None):
        x = torch.empty((self.dim, n), dtype=torch.float32, device="cuda")
        lq = torch.empty((n,), dtype=torch.float32, device="cuda")
        L.check(L.lib().fd_nsf_sample(self.handle, seed, it, inst, n, _ptr(x), _ptr(lq), _stream_ptr(stream)))
        return x, lq

    def draw(self, seed, it, inst, n, stream=None):
        """Proposals for the integrand and the chains: (x [dim][n], w = 1/q(x) [n]),
        the same stream as sample()."""
        x = torch.empty((self.dim, n), dtype=torch.float32, device="cuda")
        w = torch.empty((n,), dtype=torch.float32, device="cuda")
        L.check(L.lib().fd_nsf_sample_w(self.handle, seed, it, inst, n, _ptr(x), _ptr(w), _stream_ptr(stream)))
        return x, w

    def log_density(self, x, stream=None):
        """(z = T^-1(x), log q(x)) for device points x [dim][n]."""
        n = x.shape[1]
        assert x.dtype == torch.float32 and x.is_contiguous() and x.shape[0] == self.dim
        z = torch.empty((self.dim, n), dtype=torch.float32, device="cuda")
        lq = torch.empty((n,), dtype=torch.float32, device="cuda")
        L.check(L.lib().fd_nsf_log_density(self.handle, _ptr(x), n, _ptr(z), _ptr(lq), _stream_ptr(stream)))
        return z, lq

    def kl_grad(self, x, w, stream=None):
        """(loss, grad): the forward-KL loss -sum w log q(x) / sum w over device
        points x [dim][n] with weights w [n], and its gradient over the
        parameters (device FP64 [1], device FP32 [n_params])."""
        n = x.shape[1]
        assert x.dtype == torch.float32 and x.is_contiguous() and x.shape[0] == self.dim
        assert w.dtype == torch.float32 and w.is_contiguous() and w.shape == (n,)
        grad = torch.empty((self.n_params,), dtype=torch.float32, device="cuda")
        loss = torch.empty((1,), dtype=torch.float64, device="cuda")
        L.check(L.lib().fd_nsf_kl_grad(self.handle, _ptr(x), _ptr(w), n, _ptr(grad), _ptr(loss),
                                       _stream_ptr(stream)))
        return loss, grad

    def train(self, x, w, steps, lr, stream=None):
        """`steps` Adam steps on the batch (x, w); returns the loss before each step."""
        assert x.dtype == torch.float32 and x.is_contiguous() and x.shape[0] == self.dim
        assert w.dtype == torch.float32 and w.is_contiguous() and w.shape == (x.shape[1],)
        out = np.empty(steps, dtype=np.float64)
        L.check(L.lib().fd_nsf_train(self.handle, _ptr(x), _ptr(w), x.shape[1], steps, lr,
                                     out.ctypes.data, _stream_ptr(stream)))
        return out

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and L._lib is not None:
            L._lib.fd_nsf_free(h)
            self.handle = None


class Chains:
    """Independence Metropolis-Hastings chains over evaluated proposals (NF-MCMC
    with flow proposals, VEGAS-MCMC with VEGAS proposals; Sec. V).  Weights w
    [n_out][ld] (device FP32, e.g. EvalPlan.per_sample[inst].reshape(-1, n)):
    proposal k of chain c in column k * n_chains + c."""

    def __init__(self, n_out, n_chains, n_sel=1, alpha=0.5):
        self.n_out, self.n_chains, self.n_sel, self.alpha = n_out, n_chains, n_sel, alpha
        self.state = torch.zeros((n_out + 1, n_chains), dtype=torch.float64, device="cuda")
        self.sums = torch.zeros((n_out + 2, n_chains), dtype=torch.float64, device="cuda")
        self.out = torch.zeros((n_out + 1, 2), dtype=torch.float64, device="cuda")

    def run(self, w, n_steps, seed, it, n_therm=0, stream=None):
        """Advance every chain by n_steps (sums of this call in .sums); returns the
        estimates [n_out + 1][2]: (I, variance) per component, then (accepted fraction, 0)."""
        assert w.dtype == torch.float32 and w.is_cuda and w.dim() == 2 and w.stride(1) == 1
        assert w.shape[0] >= self.n_out
        L.check(L.lib().fd_mcmc_chains(_ptr(w), self.n_out, w.stride(0), self.n_sel, self.n_chains, n_steps,
                                       self.alpha, seed, it, n_therm, _ptr(self.state), _ptr(self.sums),
                                       _stream_ptr(stream)))
        L.check(L.lib().fd_mcmc_estimate(_ptr(self.sums), self.n_out, self.n_chains, n_steps, _ptr(self.out),
                                         _stream_ptr(stream)))
        return self.out


def measure_peak(kind):
    """Measured pipe throughput: 0 FP32 FMA (flop/s), 1 SFU ex2, 2 SFU rcp (results/s), 3 packed FP32x2 FMA (flop/s)."""
    v = ctypes.c_double()
    L.check(L.lib().fd_measure_peak(kind, ctypes.byref(v)))
    return v.value


def device_status(stream=None):
    L.check(L.lib().fd_device_status(_stream_ptr(stream)))


def set_wait_polls(polls):
    """Test hook: the interpreter's tape waits give up after `polls` polls
    (0: at once; negative: the default)."""
    L.check(L.lib().fd_debug_set_wait_polls(int(polls)))


def postprocess(N, sigma, dsigma, kF, beta, Lam):
    """Host FP64 post-process: dict (n,m,l)->complex estimates -> dmu, a, b, meff series."""
    shape = (N + 1, N + 1, N + 1)
    sre, sim, dre = np.zeros(shape), np.zeros(shape), np.zeros(shape)
    for (n, m, l), v in sigma.items():
        sre[n, m, l], sim[n, m, l] = complex(v).real, complex(v).imag
    for (n, m, l), v in dsigma.items():
        dre[n, m, l] = complex(v).real
    outs = [np.zeros(N + 1) for _ in range(4)]
    P = ctypes.POINTER(ctypes.c_double)
    L.check(L.lib().fd_postprocess(N, sre.ctypes.data_as(P), sim.ctypes.data_as(P), dre.ctypes.data_as(P), kF,
                                   beta, Lam, *[o.ctypes.data_as(P) for o in outs]))
    return dict(zip(("dmu", "a", "b", "meff"), outs))
