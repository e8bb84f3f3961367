"""Python front end of the gbnfft C ABI, on PyTorch tensors.

PyTorch provides device memory and streams only; every transform step runs in
libgbnfft.so.  Tensors on the GPU are used in place.  Tensors on the host are
copied to the GPU on the plan's stream first and the result is copied back
(the end-to-end path a caller with host data uses).

Names follow the paper (Section 1): N bandwidths (I_N), M points x_j,
adjoint = Eq. 5 (fhat(k) = sum_j f(x_j) exp(-2 pi i k.x_j)),
forward = Eq. 6 (f(x_j) = sum_k fhat(k) exp(+2 pi i k.x_j)).
"""
import ctypes

import numpy as np
import torch

from . import _lib


def _stream_handle(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Plan:
    """An NFFT plan: bandwidth N (d even ints), M points, oversampling sigma,
    cut-off m, window ("kaiser_bessel" or "gaussian"), precision ("fp32" for
    the mixed FP32 form, "fp64" for the plain FP64 form)."""

    def __init__(self, N, M, sigma=2.0, m=4, window="kaiser_bessel", precision="fp32", stream=None):
        self._lib = _lib.load()
        self.N = tuple(int(v) for v in N)
        self.d = len(self.N)
        self.M = int(M)
        self.window = _lib.WINDOWS[window] if isinstance(window, str) else int(window)
        self.precision = _lib.PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.cdtype = torch.complex128 if self.precision == _lib.FP64 else torch.complex64
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        Narr = (ctypes.c_int64 * self.d)(*self.N)
        _lib.check(self._lib.nfft_plan_create(ctypes.byref(h), self.d, Narr, self.M, float(sigma), int(m),
                                              self.window, self.precision, _stream_handle(self.stream)),
                   "nfft_plan_create")
        self._h = h
        self._x = None

    # -- lifetime -------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.nfft_plan_destroy(self._h)
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

    # -- helpers -----------------------------------------------------------------
    def _copy_stream(self):
        """Host-to-device copies run on their own stream, ordered against the
        plan's stream by events, so that they overlap kernels of earlier
        calls."""
        if getattr(self, "_cs", None) is None:
            self._cs = torch.cuda.Stream(self.device)
        return self._cs

    def _out_stream(self):
        """Device-to-host copies of results run on a third stream: a result
        waits for its own kernels only, and the next call's inputs (on the
        copy stream) do not queue behind it."""
        if getattr(self, "_os", None) is None:
            self._os = torch.cuda.Stream(self.device)
        return self._os

    def _to_device(self, t, dtype):
        if t.device.type != "cuda":
            cs = self._copy_stream()
            with torch.cuda.stream(cs):
                d = t.to(device=self.device, dtype=dtype, non_blocking=True).contiguous()
            ev = torch.cuda.Event()
            ev.record(cs)
            self.stream.wait_event(ev)
            d.record_stream(self.stream)
            return d, True
        if t.dtype != dtype:
            raise TypeError("expected %s, got %s" % (dtype, t.dtype))
        return t.contiguous(), False

    # -- C ABI calls ---------------------------------------------------------------
    def set_points(self, x):
        """x: (M, d) float64, any finite values (wrapped into [-1/2, 1/2)^d)."""
        if tuple(x.shape) != (self.M, self.d):
            raise ValueError("points must have shape (%d, %d)" % (self.M, self.d))
        xd, _ = self._to_device(x, torch.float64)
        self._x = xd  # keep alive until the sort kernels have read it
        _lib.check(self._lib.nfft_set_points(self._h, ctypes.c_void_p(xd.data_ptr())), "nfft_set_points")

    def _result_buffer(self, shape, out):
        """Device buffer for a result: `out` itself when it is a CUDA tensor,
        else a new one, kept alive for the plan's stream."""
        if out is not None and out.device.type == "cuda":
            if out.dtype != self.cdtype or out.numel() != int(np.prod(shape)):
                raise ValueError("out must hold %s %s values" % (shape, self.cdtype))
            return out
        dev = torch.empty(shape, dtype=self.cdtype, device=self.device)
        dev.record_stream(self.stream)
        return dev

    def _finish(self, dev, out, host, single):
        """A CPU `out` (pinned, for an asynchronous copy) receives the result
        on the copy stream once the plan's stream has produced it: valid after
        sync().  Otherwise a host input gets its result back as a new CPU
        tensor (a blocking copy)."""
        if out is not None and out.device.type == "cpu":
            if out.dtype != self.cdtype or out.numel() != dev.numel() or not out.is_contiguous():
                raise ValueError("out must be a contiguous tensor of %d %s values" % (dev.numel(), self.cdtype))
            res = out.view(dev.shape)
            ev = torch.cuda.Event()
            ev.record(self.stream)
            os_ = self._out_stream()
            os_.wait_event(ev)
            with torch.cuda.stream(os_):
                res.copy_(dev, non_blocking=True)
            dev.record_stream(os_)
        elif host:
            with torch.cuda.stream(self.stream):
                res = dev.to("cpu")
        else:
            res = dev.view(dev.shape)
        return res[0] if single else res

    def adjoint(self, f, out=None):
        """Eq. 5.  f: (M,) or (R, M) complex; returns N or (R,) + N complex.
        out: a CUDA tensor, or a pinned CPU tensor that receives the result
        asynchronously (read it after sync())."""
        single = f.dim() == 1
        rows = (1 if single else f.shape[0]) if self.M == 0 else -1
        fd, host = self._to_device(f.reshape(rows, self.M), self.cdtype)
        R = fd.shape[0]
        dev = self._result_buffer((R,) + self.N, out)
        _lib.check(self._lib.nfft_adjoint(self._h, ctypes.c_void_p(fd.data_ptr()), ctypes.c_void_p(dev.data_ptr()), R),
                   "nfft_adjoint")
        return self._finish(dev.view((R,) + self.N), out, host, single)

    def forward(self, fhat, out=None):
        """Eq. 6.  fhat: N or (R,) + N complex; returns (M,) or (R, M) complex.
        out: as for adjoint()."""
        single = fhat.dim() == self.d
        hd, host = self._to_device(fhat.reshape((-1,) + self.N), self.cdtype)
        R = hd.shape[0]
        dev = self._result_buffer((R, self.M), out)
        _lib.check(self._lib.nfft_forward(self._h, ctypes.c_void_p(hd.data_ptr()), ctypes.c_void_p(dev.data_ptr()), R),
                   "nfft_forward")
        return self._finish(dev.view((R, self.M)), out, host, single)

    def ewald_reciprocal(self, q, L, alpha):
        """Eq. 12 for charges q (M values) at the points set (x = r / L).
        Returns (U^K, n-sum term, self term) as floats."""
        qd, _ = self._to_device(q.reshape(self.M), self.cdtype)
        out = (ctypes.c_double * 3)()
        _lib.check(self._lib.nfft_ewald_reciprocal(self._h, ctypes.c_void_p(qd.data_ptr()), float(L), float(alpha),
                                                   out), "nfft_ewald_reciprocal")
        return out[0], out[1], out[2]

    def ewald_reciprocal_forces(self, q, L, alpha, out=None):
        """Reciprocal-space Ewald forces, the negative gradient of Eq. 12, on
        the points set (x = r / L - 1/2, 3-D): returns an (M, 3) float64 CUDA
        tensor (asynchronous on the plan's stream)."""
        qd, _ = self._to_device(q.reshape(self.M), self.cdtype)
        if out is None:
            out = torch.empty((self.M, 3), dtype=torch.float64, device=self.device)
            out.record_stream(self.stream)
        elif out.dtype != torch.float64 or out.numel() != 3 * self.M or not out.is_cuda or not out.is_contiguous():
            raise ValueError("out must be a contiguous CUDA float64 tensor of M x 3 values")
        _lib.check(self._lib.nfft_ewald_reciprocal_forces(self._h, ctypes.c_void_p(qd.data_ptr()), float(L),
                                                          float(alpha), ctypes.c_void_p(out.data_ptr())),
                   "nfft_ewald_reciprocal_forces")
        return out

    def ewald_reciprocal_sum(self, S, L, alpha, out=None):
        """The n-sum term of Eq. 12 from a structure factor S on I_N; returns
        a 1-element float64 CUDA tensor (asynchronous)."""
        Sd, _ = self._to_device(S.reshape(self.N), self.cdtype)
        if out is None:
            out = torch.empty(1, dtype=torch.float64, device=self.device)
        _lib.check(self._lib.nfft_ewald_reciprocal_sum(self._h, ctypes.c_void_p(Sd.data_ptr()), float(L), float(alpha),
                                                       ctypes.c_void_p(out.data_ptr())), "nfft_ewald_reciprocal_sum")
        return out

    def sync(self):
        """Wait for the plan's stream and its host copies; raises NFFTError for
        a device-side error."""
        for st in (getattr(self, "_cs", None), getattr(self, "_os", None)):
            if st is not None:
                st.synchronize()
        _lib.check(self._lib.nfft_sync(self._h), "nfft_sync")

    def set_option(self, option, value):
        _lib.check(self._lib.nfft_set_option(self._h, int(option), int(value)), "nfft_set_option")

    def info(self):
        inf = _lib.PlanInfo()
        _lib.check(self._lib.nfft_get_info(self._h, ctypes.byref(inf)), "nfft_get_info")
        return dict(d=inf.d, N=tuple(inf.N[:inf.d]), n=tuple(inf.n[:inf.d]), M=inf.M, m=inf.m, taps=inf.taps,
                    window=inf.window, precision=inf.precision, method=inf.method, bin=tuple(inf.bin[:inf.d]),
                    n_bins=inf.n_bins, rhs_capacity=inf.rhs_capacity, threads=inf.threads,
                    device_bytes=inf.device_bytes, sigma=tuple(inf.sigma[:inf.d]),
                    max_subproblem=inf.max_subproblem, spread_threads=inf.spread_threads,
                    sparse_points=inf.sparse_points, sparse_points_interp=inf.sparse_points_interp,
                    owner_spread=inf.owner_spread, kernel_launches=inf.kernel_launches,
                    interp_threads=inf.interp_threads, spread_block_threads=inf.spread_block_threads,
                    interp_block_threads=inf.interp_block_threads, tensor_spread=inf.tensor_spread,
                    tensor_interp=inf.tensor_interp, pruned_fft=inf.pruned_fft)

    def autotune(self, reps=3):
        """Time candidate layouts on the points set and keep the fastest;
        returns the winner's adjoint + forward milliseconds."""
        ms = ctypes.c_double()
        _lib.check(self._lib.nfft_autotune(self._h, int(reps), ctypes.byref(ms)), "nfft_autotune")
        return ms.value

    def stage_times(self, reset=False):
        """Per-stage milliseconds and call counts (needs OPT_PROFILE on)."""
        ms = (ctypes.c_double * len(_lib.STAGES))()
        n = (ctypes.c_int64 * len(_lib.STAGES))()
        _lib.check(self._lib.nfft_stage_times(self._h, ms, n, 1 if reset else 0), "nfft_stage_times")
        return {s: (ms[i], n[i]) for i, s in enumerate(_lib.STAGES)}


class Batch:
    """Many independent transforms set up once and run together (one CUDA
    graph launch per call).  items: list of dicts with keys N (tuple), M,
    and optionally sigma, m, window, nrhs."""

    def __init__(self, items, precision="fp32", stream=None, sigma=2.0, m=4, window="kaiser_bessel"):
        self._lib = _lib.load()
        self.precision = _lib.PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.cdtype = torch.complex128 if self.precision == _lib.FP64 else torch.complex64
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        arr = (_lib.BatchItem * len(items))()
        self.items = []
        for i, it in enumerate(items):
            N = tuple(int(v) for v in it["N"])
            win = it.get("window", window)
            win = _lib.WINDOWS[win] if isinstance(win, str) else int(win)
            arr[i].d = len(N)
            for t in range(3):
                arr[i].N[t] = N[t] if t < len(N) else 1
            arr[i].M = int(it["M"])
            arr[i].sigma = float(it.get("sigma", sigma))
            arr[i].m = int(it.get("m", m))
            arr[i].window = win
            arr[i].nrhs = int(it.get("nrhs", 1))
            self.items.append(dict(N=N, M=int(it["M"]), nrhs=arr[i].nrhs))
        h = ctypes.c_void_p()
        _lib.check(self._lib.nfft_batch_create(ctypes.byref(h), len(items), arr, self.precision,
                                               _stream_handle(self.stream)), "nfft_batch_create")
        self._h = h
        self._keep = []

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.nfft_batch_destroy(self._h)
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

    @staticmethod
    def _ptrs(tensors):
        return (ctypes.c_void_p * len(tensors))(*[ctypes.c_void_p(t.data_ptr()) for t in tensors])

    def set_points(self, xs):
        """xs: list of (M_i, d_i) float64 CUDA tensors."""
        xs = [x.contiguous() for x in xs]
        self._x = xs
        _lib.check(self._lib.nfft_batch_set_points(self._h, self._ptrs(xs)), "nfft_batch_set_points")

    def adjoint(self, fs, outs=None):
        """Eq. 5 for every item: fs[i] (nrhs_i, M_i) complex -> (nrhs_i,) + N_i."""
        fs = [f.contiguous() for f in fs]
        if outs is None:
            outs = [torch.empty((it["nrhs"],) + it["N"], dtype=self.cdtype, device=self.device) for it in self.items]
        self._keep = [fs, outs]
        _lib.check(self._lib.nfft_batch_adjoint(self._h, self._ptrs(fs), self._ptrs(outs)), "nfft_batch_adjoint")
        return outs

    def forward(self, fhats, outs=None):
        """Eq. 6 for every item: fhats[i] (nrhs_i,) + N_i -> (nrhs_i, M_i)."""
        fhats = [h.contiguous() for h in fhats]
        if outs is None:
            outs = [torch.empty((it["nrhs"], it["M"]), dtype=self.cdtype, device=self.device) for it in self.items]
        self._keep = [fhats, outs]
        _lib.check(self._lib.nfft_batch_forward(self._h, self._ptrs(fhats), self._ptrs(outs)), "nfft_batch_forward")
        return outs

    def sync(self):
        _lib.check(self._lib.nfft_batch_sync(self._h), "nfft_batch_sync")

    def autotune(self, reps=3):
        ms = ctypes.c_double()
        _lib.check(self._lib.nfft_batch_autotune(self._h, int(reps), ctypes.byref(ms)), "nfft_batch_autotune")
        return ms.value

    def set_option(self, option, value):
        _lib.check(self._lib.nfft_batch_set_option(self._h, int(option), int(value)), "nfft_batch_set_option")

    def kernel_launches(self):
        """This library's kernels launched by the batch so far."""
        c = ctypes.c_int64()
        _lib.check(self._lib.nfft_batch_kernel_launches(self._h, ctypes.byref(c)), "nfft_batch_kernel_launches")
        return c.value

    def stage_times(self, reset=False):
        ms = (ctypes.c_double * len(_lib.STAGES))()
        n = (ctypes.c_int64 * len(_lib.STAGES))()
        _lib.check(self._lib.nfft_batch_stage_times(self._h, ms, n, 1 if reset else 0), "nfft_batch_stage_times")
        return {s: (ms[i], n[i]) for i, s in enumerate(_lib.STAGES)}


def plan_params(N, sigma=2.0, m=4, window="kaiser_bessel"):
    """Host-only rule: oversampled sizes n_t and window taps per dimension."""
    lib = _lib.load()
    d = len(N)
    Narr = (ctypes.c_int64 * d)(*[int(v) for v in N])
    nout = (ctypes.c_int64 * d)()
    taps = ctypes.c_int()
    win = _lib.WINDOWS[window] if isinstance(window, str) else int(window)
    _lib.check(lib.nfft_plan_params(d, Narr, float(sigma), int(m), win, nout, ctypes.byref(taps)), "nfft_plan_params")
    return tuple(nout), taps.value


def ewald_real_space(r, q, L, alpha, rcut, stream=None):
    """Eq. 11: the real-space Ewald energy of charges q (n) at positions r
    (n x 3, any finite values, periodic box of edge L), pairs and images
    closer than rcut (0 < rcut < L).  CPU tensors are copied to the device
    first.  Waits for the stream and returns the energy as a float."""
    lib = _lib.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    with torch.cuda.stream(st):
        rd = r.to(device=dev, dtype=torch.float64).contiguous()
        qd = q.to(device=dev, dtype=torch.float64).contiguous()
    if rd.dim() != 2 or rd.shape[1] != 3 or qd.numel() != rd.shape[0]:
        raise ValueError("r must be (n, 3) and q must hold n charges")
    out = ctypes.c_double()
    _lib.check(lib.nfft_ewald_real_space(int(rd.shape[0]), ctypes.c_void_p(rd.data_ptr()),
                                         ctypes.c_void_p(qd.data_ptr()), float(L), float(alpha), float(rcut),
                                         ctypes.byref(out), _stream_handle(st)), "nfft_ewald_real_space")
    return out.value


def ewald_real_space_forces(r, q, L, alpha, rcut, stream=None):
    """The negative gradient of Eq. 11: forces (n x 3 float64 CUDA tensor) and
    the real-space energy (float) of charges q at positions r, pairs and
    images closer than rcut (0 < rcut < L).  Waits for the stream."""
    lib = _lib.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    with torch.cuda.stream(st):
        rd = r.to(device=dev, dtype=torch.float64).contiguous()
        qd = q.to(device=dev, dtype=torch.float64).contiguous()
        F = torch.empty((rd.shape[0], 3), dtype=torch.float64, device=dev)
    if rd.dim() != 2 or rd.shape[1] != 3 or qd.numel() != rd.shape[0]:
        raise ValueError("r must be (n, 3) and q must hold n charges")
    e = ctypes.c_double()
    _lib.check(lib.nfft_ewald_real_space_forces(int(rd.shape[0]), ctypes.c_void_p(rd.data_ptr()),
                                                ctypes.c_void_p(qd.data_ptr()), float(L), float(alpha), float(rcut),
                                                ctypes.c_void_p(F.data_ptr()), ctypes.byref(e), _stream_handle(st)),
               "nfft_ewald_real_space_forces")
    return F, e.value
