"""qvx: single amplitudes <x|C|0...0> by variable elimination with slicing, on GB300.

Python binding of libqvx.so (include/qvx.h). It only marshals arguments: circuits into
qvx_gate arrays, torch tensors into device pointers and the caller's current CUDA stream
into the stream argument. Every step of the computation runs in the library's kernels;
if the library is missing the binding raises, it never falls back to another path.

    plan = Plan(circuit, n_slices=12)          # host planner (Sections 3.A-3.B)
    amps = plan.amplitude(bitstrings)          # complex128 torch tensor on the device
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqvx.so")

QVX_OK, QVX_EINVAL, QVX_ENOMEM, QVX_ECUDA, QVX_ETIMEOUT, QVX_EUNSUPPORTED, QVX_ERANGE = range(7)
ENGINES = {"auto": 0, "fused": 1, "stepwise": 2, "persistent": 3}
ENGINE_NAMES = {v: k for k, v in ENGINES.items()}


class QvxError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"qvx status {status}: {msg}")
        self.status = status


class Gate(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("q0", ctypes.c_int32), ("q1", ctypes.c_int32),
                ("param_index", ctypes.c_int32), ("theta", ctypes.c_double), ("phi", ctypes.c_double),
                ("u", ctypes.c_double * 8)]


class CircuitStruct(ctypes.Structure):
    _fields_ = [("n_qubits", ctypes.c_int32), ("reserved", ctypes.c_int32), ("n_gates", ctypes.c_int64),
                ("gates", ctypes.POINTER(Gate))]


class PlanOpts(ctypes.Structure):
    _fields_ = [("n_slices", ctypes.c_int32), ("order_restarts", ctypes.c_int32),
                ("order_seed", ctypes.c_uint64), ("mem_budget_bytes", ctypes.c_int64),
                ("engine", ctypes.c_int32), ("inner_slices", ctypes.c_int32),
                ("max_rank", ctypes.c_int32), ("warps_per_item", ctypes.c_int32),
                ("host_merge_rank", ctypes.c_int32), ("gradient", ctypes.c_int32),
                ("slice_rule", ctypes.c_int32), ("n_open_qubits", ctypes.c_int32),
                ("open_qubits", ctypes.c_int32 * 16), ("tensor_cores", ctypes.c_int32),
                ("plan_trials", ctypes.c_int32)]


class PlanInfo(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("n_qubits", "n_vars", "n_edges", "n_sliced", "n_inner",
                                               "n_steps", "n_leaves", "max_rank", "engine",
                                               "warps_per_item")] + \
               [("n_items_per_bitstring", ctypes.c_int64), ("log2_cost", ctypes.c_double),
                ("log2_cost_unsliced", ctypes.c_double), ("flops_per_amplitude", ctypes.c_double),
                ("bytes_per_amplitude", ctypes.c_double), ("arena_bytes", ctypes.c_int64),
                ("device_image_bytes", ctypes.c_int64), ("n_params", ctypes.c_int32),
                ("n_grad_steps", ctypes.c_int32), ("grad_arena_bytes", ctypes.c_int64),
                ("grad_flops_per_amplitude", ctypes.c_double), ("grad_bytes_per_amplitude", ctypes.c_double),
                ("n_tiled_steps", ctypes.c_int32), ("n_phases", ctypes.c_int32),
                ("n_open_qubits", ctypes.c_int32), ("n_gemm_steps", ctypes.c_int32),
                ("grad_smem_bytes", ctypes.c_int32), ("grad_recomputed", ctypes.c_int32),
                ("est_bytes_per_amplitude", ctypes.c_double)]


class LaunchRecord(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int32), ("step", ctypes.c_int32), ("items", ctypes.c_int64),
                ("flops", ctypes.c_double), ("bytes", ctypes.c_double), ("ms", ctypes.c_float),
                ("pad", ctypes.c_int32)]


_lib = None
EXPORTED = ("qvx_plan_opts_default", "qvx_graph_export", "qvx_plan_create", "qvx_plan_destroy",
            "qvx_plan_get_info", "qvx_plan_get_order", "qvx_plan_get_image", "qvx_workspace_size", "qvx_workspace_init",
            "qvx_amplitude", "qvx_amplitude_slices", "qvx_slice_terms", "qvx_workspace_status",
            "qvx_last_error", "qvx_amplitude_noalloc", "qvx_amplitude_grad", "qvx_amplitude_host",
            "qvx_selftest_wait_timeout", "qvx_kernel_launches", "qvx_noalloc_status", "qvx_amplitude_profiled",
            "qvx_profile_read", "qvx_kernel_name", "qvx_selftest_fused_timeout")


def lib():
    """The loaded libqvx.so; raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    P, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
    sig = {
        "qvx_plan_opts_default": (None, [ctypes.POINTER(PlanOpts)]),
        "qvx_graph_export": (ctypes.c_int, [ctypes.POINTER(CircuitStruct), P, P, P, P, P, i64]),
        "qvx_plan_create": (ctypes.c_int, [ctypes.POINTER(CircuitStruct), P, i32, P, i32,
                                           ctypes.POINTER(PlanOpts), ctypes.POINTER(P)]),
        "qvx_plan_destroy": (None, [P]),
        "qvx_plan_get_info": (ctypes.c_int, [P, ctypes.POINTER(PlanInfo)]),
        "qvx_plan_get_order": (ctypes.c_int, [P, P, P]),
        "qvx_plan_get_image": (ctypes.c_int, [P, ctypes.POINTER(P), ctypes.POINTER(ctypes.c_size_t)]),
        "qvx_workspace_size": (ctypes.c_int, [P, i64, ctypes.POINTER(ctypes.c_size_t)]),
        "qvx_workspace_init": (ctypes.c_int, [P, P, ctypes.c_size_t, P]),
        "qvx_amplitude": (ctypes.c_int, [P, P, i64, P, P, ctypes.c_size_t, P]),
        "qvx_amplitude_slices": (ctypes.c_int, [P, P, i64, i64, i64, P, P, ctypes.c_size_t, P]),
        "qvx_slice_terms": (ctypes.c_int, [P, P, i64, i64, i64, P, P, ctypes.c_size_t, P]),
        "qvx_workspace_status": (ctypes.c_int, [P, P, P]),
        "qvx_last_error": (ctypes.c_char_p, []),
        "qvx_kernel_launches": (ctypes.c_uint64, []),
        "qvx_amplitude_noalloc": (ctypes.c_int, [P, P, i64, P, P]),
        "qvx_amplitude_grad": (ctypes.c_int, [P, P, i64, P, i32, P, P, P, ctypes.c_size_t, P]),
        "qvx_amplitude_host": (ctypes.c_int, [P, P, i64, P, P, ctypes.c_size_t, P]),
        "qvx_selftest_wait_timeout": (ctypes.c_int, [P, P, ctypes.c_size_t, ctypes.c_uint32, P]),
        "qvx_noalloc_status": (ctypes.c_int, [P]),
        "qvx_amplitude_profiled": (ctypes.c_int, [P, P, i64, i64, i64, P, P, ctypes.c_size_t, P]),
        "qvx_profile_read": (ctypes.c_int, [P, ctypes.POINTER(LaunchRecord), i64, ctypes.POINTER(ctypes.c_int64)]),
        "qvx_kernel_name": (ctypes.c_char_p, [i32]),
        "qvx_selftest_fused_timeout": (ctypes.c_int, [P, P, i64, P, P, ctypes.c_size_t, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    del u64
    _lib = L
    return L


def _check(status):
    if status != QVX_OK:
        raise QvxError(status, lib().qvx_last_error().decode(errors="replace"))


def circuit_struct(circ):
    """qvx_circuit for a circuitgen.Circuit-like object (n_qubits, gates with kind/q0/q1/...)."""
    n = len(circ.gates)
    arr = (Gate * max(n, 1))()
    for i, g in enumerate(circ.gates):
        arr[i].kind, arr[i].q0, arr[i].q1 = g.kind, g.q0, g.q1
        arr[i].param_index = getattr(g, "param", -1)
        arr[i].theta, arr[i].phi = getattr(g, "theta", 0.0), getattr(g, "phi", 0.0)
        u = getattr(g, "u", ())
        for j in range(len(u)):
            arr[i].u[j] = u[j]
    cs = CircuitStruct(circ.n_qubits, 0, n, ctypes.cast(arr, ctypes.POINTER(Gate)))
    cs._keep = arr
    return cs


def graph_export(circ):
    """(var_qubit, var_ordinal, edges) of the circuit's graphical model (Section 3.A)."""
    L = lib()
    cs = circuit_struct(circ)
    nv, ne = ctypes.c_int32(), ctypes.c_int64()
    _check(L.qvx_graph_export(ctypes.byref(cs), ctypes.byref(nv), None, None, ctypes.byref(ne), None, 0))
    vq = (ctypes.c_int32 * max(nv.value, 1))()
    vo = (ctypes.c_int32 * max(nv.value, 1))()
    ed = (ctypes.c_int32 * max(2 * ne.value, 1))()
    _check(L.qvx_graph_export(ctypes.byref(cs), None, vq, vo, None, ed, ne.value))
    return (list(vq[:nv.value]), list(vo[:nv.value]),
            [(ed[2 * i], ed[2 * i + 1]) for i in range(ne.value)])


def bitstring_words(bitstrings, words):
    """Python ints (bit q = qubit q) as the int64 words of the C interface: `words` words per
    bitstring, bit q in word q // 64 (two's-complement views of the unsigned words)."""
    out = []
    for b in bitstrings:
        v = int(b)
        for w in range(words):
            u = (v >> (64 * w)) & ((1 << 64) - 1)
            out.append(u - (1 << 64) if u >= 1 << 63 else u)
    return out


def bits_tensor(bitstrings, words, device=None):
    """A contiguous int64 device tensor of `words` words per bitstring, from a tensor (already
    in that layout) or from Python ints."""
    import torch
    if isinstance(bitstrings, torch.Tensor):
        t = bitstrings
        if t.dtype != torch.int64:
            raise TypeError("bitstrings must be int64 words")
        if t.numel() % words:
            raise QvxError(QVX_EINVAL, f"bitstring words: a multiple of {words} expected")
    else:
        t = torch.tensor(bitstring_words(bitstrings, words), dtype=torch.int64)
    if not t.is_cuda:
        t = t.to(device if device is not None else "cuda")
    return t.contiguous().view(-1)


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Plan:
    """A host plan: graph, elimination order, slices and the pairwise contraction program."""

    def __init__(self, circ, order=None, slices=None, n_slices=-1, engine="auto", inner_slices=-1,
                 order_restarts=8, order_seed=1, mem_budget_bytes=1 << 30, max_rank=30,
                 warps_per_item=1, host_merge_rank=8, gradient=False, slice_rule="greedy", open_qubits=(),
                 tensor_cores=False, plan_trials=1):
        L = lib()
        opts = PlanOpts()
        L.qvx_plan_opts_default(ctypes.byref(opts))
        opts.n_slices = n_slices
        opts.order_restarts = order_restarts
        opts.order_seed = order_seed
        opts.mem_budget_bytes = mem_budget_bytes
        opts.engine = ENGINES[engine]
        opts.inner_slices = inner_slices
        opts.max_rank = max_rank
        opts.warps_per_item = warps_per_item
        opts.host_merge_rank = host_merge_rank
        opts.gradient = 1 if gradient else 0
        opts.slice_rule = {"greedy": 0, "reorder": 1, "cz-pair": 2}[slice_rule]
        opts.tensor_cores = 1 if tensor_cores else 0
        opts.plan_trials = plan_trials
        opts.n_open_qubits = len(open_qubits)
        for i, qb in enumerate(open_qubits):
            opts.open_qubits[i] = qb
        cs = circuit_struct(circ)
        o_arr = (ctypes.c_int32 * max(len(order or []), 1))(*(order or []))
        s_arr = (ctypes.c_int32 * max(len(slices or []), 1))(*(slices or []))
        h = ctypes.c_void_p()
        _check(L.qvx_plan_create(ctypes.byref(cs), o_arr, len(order or []), s_arr,
                                 -1 if slices is None else len(slices), ctypes.byref(opts),
                                 ctypes.byref(h)))
        self._h = h
        self.n_qubits = circ.n_qubits
        self.words = (circ.n_qubits + 63) // 64   # int64 words per bitstring
        inf = PlanInfo()
        _check(L.qvx_plan_get_info(h, ctypes.byref(inf)))
        self.info = {f[0]: getattr(inf, f[0]) for f in PlanInfo._fields_}
        self.info["engine"] = ENGINE_NAMES[self.info["engine"]]
        nv, k = inf.n_vars, inf.n_sliced
        o = (ctypes.c_int32 * max(nv - k, 1))()
        s = (ctypes.c_int32 * max(k, 1))()
        _check(L.qvx_plan_get_order(h, o, s))
        self.order = list(o[:nv - k])
        self.slices = list(s[:k])
        self.open_qubits = list(open_qubits)
        self.n_open = len(self.open_qubits)
        self.plan_trials = plan_trials
        self.mem_budget_bytes = mem_budget_bytes
        self._ws = {}

    def items_in_flight(self, batch):
        """Work items one pass of the global-arena engines holds (the arena budget's share)."""
        total = max(batch, 1) * self.info["n_items_per_bitstring"]
        return min(total, max(1, self.mem_budget_bytes // max(self.info["arena_bytes"], 32)))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.qvx_plan_destroy(h)
            self._h = None

    def image(self) -> bytes:
        """A copy of the plan's device image (program, leaves, element maps)."""
        p, n = ctypes.c_void_p(), ctypes.c_size_t()
        _check(lib().qvx_plan_get_image(self._h, ctypes.byref(p), ctypes.byref(n)))
        return ctypes.string_at(p, n.value)

    @property
    def n_slice_terms(self) -> int:
        return 1 << len(self.slices)

    def workspace_bytes(self, batch: int) -> int:
        n = ctypes.c_size_t()
        _check(lib().qvx_workspace_size(self._h, batch, ctypes.byref(n)))
        return n.value

    def workspace(self, batch: int, device=None, stream=None):
        """A device workspace (torch uint8) sized for `batch` bitstrings, initialised."""
        import torch
        dev = torch.device(device if device is not None else "cuda")
        nbytes = self.workspace_bytes(batch)
        buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
        shift = (-buf.data_ptr()) % 256
        ws = buf[shift:shift + nbytes]
        _check(lib().qvx_workspace_init(self._h, ctypes.c_void_p(ws.data_ptr()), nbytes, _stream_ptr(stream)))
        return ws

    def _ws_for(self, batch, device):
        key = (batch, str(device))
        if key not in self._ws:
            self._ws[key] = self.workspace(batch, device)
        return self._ws[key]

    def _bits(self, bitstrings, device=None):
        return bits_tensor(bitstrings, self.words, device)

    def _check_bits(self, bits):
        import torch
        w = bits.view(-1, self.words)
        for j in range(self.words):
            valid = self.n_qubits - 64 * j
            if valid < 64 and bool(torch.any((w[:, j] >> valid) != 0)):
                raise QvxError(QVX_EINVAL, "bitstring has bits at or above n_qubits")

    def amplitude(self, bitstrings, workspace=None, out=None, stream=None, slice_begin=0,
                  slice_count=None, validate=True):
        """<x|C|0> for each bitstring: complex128 torch tensor on the bitstrings' device.
        slice_begin/slice_count restrict the sum to a range of slice numbers."""
        import torch
        bits = self._bits(bitstrings)
        if validate:
            self._check_bits(bits)
        n = bits.numel() // self.words
        ws = workspace if workspace is not None else self._ws_for(n, bits.device)
        m = 1 << self.n_open
        if out is None:
            out = torch.empty(2 * n * m, dtype=torch.float64, device=bits.device)
        if slice_count is None:
            slice_count = self.n_slice_terms - slice_begin
        _check(lib().qvx_amplitude_slices(self._h, ctypes.c_void_p(bits.data_ptr()), n, slice_begin,
                                          slice_count, ctypes.c_void_p(out.data_ptr()),
                                          ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream_ptr(stream)))
        a = torch.view_as_complex(out.view(n * m, 2))
        return a.view(n, m) if self.n_open else a

    def amplitude_grad(self, bitstrings, thetas=None, workspace=None, stream=None):
        """(alpha [batch] complex128, d alpha / d theta [batch, n_params] complex128) on the
        device, for a plan created with gradient=True. thetas: float64 tensor of n_params
        angles (any device) replacing the circuit's, or None."""
        import torch
        bits = self._bits(bitstrings)
        self._check_bits(bits)
        n = bits.numel() // self.words
        npar = self.info["n_params"]
        ws = workspace if workspace is not None else self._ws_for(n, bits.device)
        amps = torch.empty(2 * n, dtype=torch.float64, device=bits.device)
        grad = torch.empty(2 * n * max(npar, 1), dtype=torch.float64, device=bits.device)
        th = None
        if thetas is not None:
            th = torch.as_tensor(thetas, dtype=torch.float64).to(bits.device).contiguous()
            if th.numel() != npar:
                raise QvxError(QVX_EINVAL, f"expected {npar} angles, got {th.numel()}")
        _check(lib().qvx_amplitude_grad(self._h, ctypes.c_void_p(bits.data_ptr()), n,
                                        None if th is None else ctypes.c_void_p(th.data_ptr()),
                                        0 if th is None else npar, ctypes.c_void_p(amps.data_ptr()),
                                        ctypes.c_void_p(grad.data_ptr()), ctypes.c_void_p(ws.data_ptr()),
                                        ws.numel(), _stream_ptr(stream)))
        a = torch.view_as_complex(amps.view(n, 2))
        g = torch.view_as_complex(grad.view(n, max(npar, 1), 2))[:, :npar]
        return a, g

    def graphed(self, bitstrings, workspace=None):
        """Captures one amplitude call for these device bitstrings into a CUDA graph.

        Returns (replay, out): replay() re-launches every kernel of the call with one graph
        launch on the current stream; out (complex128, on the device) holds the amplitudes
        after each replay. Change the bitstrings by writing into the same device tensor.
        The call is made once outside the capture first, so the library's one-time launch
        set-up is not captured."""
        import torch
        bits = self._bits(bitstrings)
        n = bits.numel() // self.words
        ws = workspace if workspace is not None else self._ws_for(n, bits.device)
        out = torch.empty(2 * n * (1 << self.n_open), dtype=torch.float64, device=bits.device)
        side = torch.cuda.Stream(device=bits.device)
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            self.amplitude(bits, workspace=ws, out=out, validate=False, stream=side)
        torch.cuda.current_stream().wait_stream(side)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.amplitude(bits, workspace=ws, out=out, validate=False)
        self._graph_keep = (bits, ws)
        a = torch.view_as_complex(out.view(n << self.n_open, 2))
        return g.replay, (a.view(n, 1 << self.n_open) if self.n_open else a)

    def amplitude_host(self, bitstrings, out=None, workspace=None, stream=None):
        """<x|C|0> from host bitstrings into host memory (numpy complex128), blocking.
        bitstrings: a CPU int64 tensor (pinned: read by the kernel directly) or a list;
        out: an optional CPU float64 tensor of 2*batch (pinned: written directly)."""
        import torch
        if isinstance(bitstrings, torch.Tensor):
            h = bitstrings
        else:
            h = torch.tensor(bitstring_words(bitstrings, self.words), dtype=torch.int64)
        if h.is_cuda or h.dtype != torch.int64:
            raise TypeError("bitstrings must be a CPU int64 tensor or a list")
        h = h.contiguous()
        n = h.numel() // self.words
        if out is None:
            out = torch.empty(2 * n * (1 << self.n_open), dtype=torch.float64)
        dev = torch.device("cuda", torch.cuda.current_device())
        ws = workspace if workspace is not None else self._ws_for(n, dev)
        _check(lib().qvx_amplitude_host(self._h, ctypes.c_void_p(h.data_ptr()), n, ctypes.c_void_p(out.data_ptr()),
                                        ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream_ptr(stream)))
        a = out[0::2].numpy() + 1j * out[1::2].numpy()
        return a.reshape(n, 1 << self.n_open) if self.n_open else a

    def slice_terms(self, bitstrings, slice_begin=0, slice_count=None, workspace=None, stream=None):
        """The slice terms beta_s (complex64, [batch, slice_count]) of Section 3.B.2."""
        import torch
        bits = self._bits(bitstrings)
        self._check_bits(bits)
        n = bits.numel() // self.words
        if slice_count is None:
            slice_count = self.n_slice_terms - slice_begin
        ws = workspace if workspace is not None else self._ws_for(n, bits.device)
        m = 1 << self.n_open
        out = torch.empty(2 * n * m * slice_count, dtype=torch.float32, device=bits.device)
        _check(lib().qvx_slice_terms(self._h, ctypes.c_void_p(bits.data_ptr()), n, slice_begin, slice_count,
                                     ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(ws.data_ptr()),
                                     ws.numel(), _stream_ptr(stream)))
        t = torch.view_as_complex(out.view(n * m, slice_count, 2))
        return t.view(n, m, slice_count) if self.n_open else t.view(n, slice_count)

    def amplitude_profiled(self, bits, workspace, out, stream=None, slice_begin=0, slice_count=None):
        """plan.amplitude (device int64 bitstring words, caller's workspace and float64
        output) with a CUDA event before and after every kernel launch, appended to the plan's
        launch log (read_profile). Does not synchronise."""
        if slice_count is None:
            slice_count = self.n_slice_terms - slice_begin
        _check(lib().qvx_amplitude_profiled(self._h, ctypes.c_void_p(bits.data_ptr()), bits.numel() // self.words,
                                            slice_begin, slice_count, ctypes.c_void_p(out.data_ptr()),
                                            ctypes.c_void_p(workspace.data_ptr()), workspace.numel(),
                                            _stream_ptr(stream)))

    def read_profile(self):
        """The launch log of amplitude_profiled calls since the last read, in issue order: a
        list of dicts (kernel name, step, items, algorithmic flops and bytes, ms); empties it."""
        L = lib()
        n = ctypes.c_int64()
        _check(L.qvx_profile_read(self._h, None, 0, ctypes.byref(n)))   # the count; the log stays
        cap = max(n.value, 1)
        recs = (LaunchRecord * cap)()
        _check(L.qvx_profile_read(self._h, recs, cap, ctypes.byref(n)))
        return [dict(kernel=L.qvx_kernel_name(r.kernel).decode(), step=r.step, items=r.items, flops=r.flops,
                     bytes=r.bytes, ms=r.ms) for r in recs[:min(n.value, cap)]]

    def check_status(self, workspace, stream=None):
        """Synchronises and raises if a kernel set the workspace's device status word."""
        _check(lib().qvx_workspace_status(self._h, ctypes.c_void_p(workspace.data_ptr()), _stream_ptr(stream)))
