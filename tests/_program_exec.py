"""Host interpreter of a plan's device image, in complex128 (test helper).

It reads the structs of csrc/device_program.h with numpy and executes the pairwise
program exactly as the kernels define it, so the planner's program (layouts, address
runs, leaf maps, slice numbering) is checked on the CPU against the oracle. It shares no
arithmetic with the oracle: the oracle eliminates variables from its own graph.
"""
import numpy as np

RUN = np.dtype([("src", "u1"), ("len", "u1"), ("dst", "u1"), ("pad", "u1")])
STEP = np.dtype([("a_off", "<u8"), ("b_off", "<u8"), ("c_off", "<u8"), ("rc", "u1"), ("nk_ab", "u1"),
                 ("nk_a", "u1"), ("nk_b", "u1"), ("a_cb", "u1"), ("b_cb", "u1"), ("na_runs", "u1"),
                 ("nb_runs", "u1"), ("flags", "<u4"), ("pad", "<u4"), ("runs_a", RUN, (12,)),
                 ("runs_b", RUN, (12,))])
LEAF = np.dtype([("data_off", "<u4"), ("n_elem", "<u4"), ("n_fixed", "<u4"), ("pad", "<u4"),
                 ("fixed_src", "u1", (12,)), ("fixed_pos", "u1", (12,))])
PROG = np.dtype([("magic", "<u4"), ("n_steps", "<u4"), ("n_leaves", "<u4"), ("pad0", "<u4"),
                 ("n_leaf_entries", "<u8"),
                 ("arena_elems", "<u8"), ("final_off", "<u8"), ("n_inner", "<u4"),
                 ("final_present", "<u4"), ("zero_mask", "<u8"), ("scalar_re", "<f8"),
                 ("scalar_im", "<f8"), ("n_outer", "<u8"), ("steps_off", "<u8"), ("leaves_off", "<u8"),
                 ("leaf_data_off", "<u8"), ("fused_steps_off", "<u8"), ("fused_tab_off", "<u8"),
                 ("n_tab_entries", "<u8"), ("fused_lane_map_off", "<u8"), ("n_fused_phases", "<u4"),
                 ("fused_lanes", "<u4"), ("grad_steps_off", "<u8"), ("params_off", "<u8"),
                 ("codes_off", "<u8"), ("deriv_data_off", "<u8"), ("thetas_off", "<u8"),
                 ("param_csr_off", "<u8"), ("n_grad_steps", "<u4"), ("n_param_leaves", "<u4"),
                 ("n_params", "<u4"), ("grad_pad", "<u4"), ("grad_arena_elems", "<u8"),
                 ("final_fwd_off", "<u8"), ("gslot_off", "<u8"), ("level_phases_off", "<u8"),
                 ("n_level_phases", "<u4"), ("n_grad_phases", "<u4"), ("grad_phases_off", "<u8"),
                 ("grad_elem_off_off", "<u8"), ("n_open", "<u4"), ("open_present", "<u4"),
                 ("regtile_off", "<u8"), ("gentry_off", "<u8"), ("gktab_off", "<u8"),
                 ("gphase_entry_off", "<u8"), ("gemm_off", "<u8"), ("image_bytes", "<u8"),
                 ("zero_mask_hi", "<u8")])
FSTEP = np.dtype([("a_off", "<u4"), ("b_off", "<u4"), ("c_off", "<u4"), ("tab_off", "<u4"), ("flags", "<u4"),
                  ("rc", "u1"), ("nk_ab", "u1"), ("nk_a", "u1"), ("nk_b", "u1"), ("a_cb", "u1"), ("b_cb", "u1"),
                  ("nk", "u1"), ("pad1", "u1"), ("pad2", "<u4"), ("koff_a", "<u2", (8,)), ("koff_b", "<u2", (8,))])
GOP = np.dtype([("off", "<u8"), ("kind", "<u4"), ("n_oruns", "u1"), ("n_kruns", "u1"), ("pad0", "u1"),
                ("pad1", "u1"), ("oruns", RUN, (12,)), ("kruns", RUN, (12,))])
GSTEP = np.dtype([("x", GOP), ("y", GOP), ("out_off", "<u8"), ("ro", "<u4"), ("nk", "<u4")])
PLEAF = np.dtype([("leaf", "<u4"), ("param", "<u4"), ("n_stored", "<u4"), ("code_off", "<u4"), ("phi", "<f8")])
RTSTEP = np.dtype([("a_off", "<u8"), ("b_off", "<u8"), ("c_off", "<u8"), ("flags", "<u4"), ("rc", "u1"),
                   ("nt", "u1"), ("rm", "u1"), ("rn", "u1"), ("nk_ab", "u1"), ("nk_a", "u1"), ("nk_b", "u1"),
                   ("a_cb", "u1"), ("b_cb", "u1"), ("n_free", "u1"), ("na_runs", "u1"), ("nb_runs", "u1"),
                   ("free_runs", RUN, (6,)), ("runs_a", RUN, (12,)), ("runs_b", RUN, (12,)),
                   ("a_m", "<u4", (8,)), ("b_n", "<u4", (8,)), ("c_m", "<u4", (8,)), ("c_n", "<u4", (8,))])
assert STEP.itemsize == 136 and LEAF.itemsize == 40 and PROG.itemsize == 328 and FSTEP.itemsize == 64
GEMM = np.dtype([("a_off", "<u8"), ("b_off", "<u8"), ("c_off", "<u8"), ("flags", "<u4"), ("nb", "u1"),
                 ("nm", "u1"), ("nn", "u1"), ("nk", "u1"), ("n_ab", "u1"), ("n_am", "u1"), ("n_ak", "u1"),
                 ("n_bb", "u1"), ("n_bn", "u1"), ("n_bk", "u1"), ("n_cb", "u1"), ("n_cm", "u1"), ("n_cn", "u1"),
                 ("pad", "u1", (3,))] + [(f, RUN, (8,)) for f in ("ab", "am", "ak", "bb", "bn", "bk", "cb", "cm", "cn")] +
                [("tail", "<u4")])
GENTRY = np.dtype([("c", "<u2"), ("meta", "<u2"), ("xr", "<u2"), ("xo", "<u2"), ("yr", "<u2"), ("yo", "<u2"),
                   ("k1", "<u4")])
assert RTSTEP.itemsize == 288 and GENTRY.itemsize == 16 and GEMM.itemsize == 336
assert GOP.itemsize == 112 and GSTEP.itemsize == 240 and PLEAF.itemsize == 24
OP_ARENA, OP_LEAF, OP_DERIV, OP_ONE = 0, 1, 2, 3
UNARY, A_LEAF, B_LEAF = 1, 2, 4


def _bf16(v):
    """float32 array rounded to bf16 (nearest even), returned as float32."""
    u = np.asarray(v, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32)


def _pext(c, runs, n):
    r = np.zeros_like(c)
    for i in range(n):
        src, ln, dst = int(runs[i]["src"]), int(runs[i]["len"]), int(runs[i]["dst"])
        r |= ((c >> src) & ((1 << ln) - 1)) << dst
    return r


class Program:
    def __init__(self, image: bytes):
        buf = np.frombuffer(image, dtype=np.uint8)
        self.h = np.frombuffer(buf[:PROG.itemsize].tobytes(), dtype=PROG)[0]
        h = self.h
        assert int(h["magic"]) == 0x51565831
        self.steps = np.frombuffer(buf[int(h["steps_off"]):int(h["steps_off"]) + STEP.itemsize * int(h["n_steps"])].tobytes(), dtype=STEP)
        self.leaves = np.frombuffer(buf[int(h["leaves_off"]):int(h["leaves_off"]) + LEAF.itemsize * int(h["n_leaves"])].tobytes(), dtype=LEAF)
        self.fsteps = None
        if int(h["fused_steps_off"]):
            fo, to = int(h["fused_steps_off"]), int(h["fused_tab_off"])
            self.fsteps = np.frombuffer(buf[fo:fo + FSTEP.itemsize * int(h["n_steps"])].tobytes(), dtype=FSTEP)
            self.tab = np.frombuffer(buf[to:to + 4 * int(h["n_tab_entries"])].tobytes(), dtype="<u4").astype(np.int64)
            lo, nl = int(h["fused_lane_map_off"]), int(h["n_fused_phases"]) * int(h["fused_lanes"])
            self.lane_map = np.frombuffer(buf[lo:lo + 4 * nl].tobytes(), dtype="<u4").reshape(
                int(h["n_fused_phases"]), int(h["fused_lanes"]))
        self.gemms = None
        if int(h["gemm_off"]):
            go = int(h["gemm_off"])
            self.gemms = np.frombuffer(buf[go:go + GEMM.itemsize * int(h["n_steps"])].tobytes(), dtype=GEMM)
        self.rtsteps = None
        if int(h["regtile_off"]):
            ro = int(h["regtile_off"])
            self.rtsteps = np.frombuffer(buf[ro:ro + RTSTEP.itemsize * int(h["n_steps"])].tobytes(), dtype=RTSTEP)
        n = int(h["n_leaf_entries"])
        ld = np.frombuffer(buf[int(h["leaf_data_off"]):int(h["leaf_data_off"]) + 8 * n].tobytes(), dtype="<f4")
        self.leaf_data = ld[0::2].astype(np.float64) + 1j * ld[1::2].astype(np.float64)
        self.gsteps = None
        if int(h["n_grad_steps"]):
            go = int(h["grad_steps_off"])
            self.gsteps = np.frombuffer(buf[go:go + GSTEP.itemsize * int(h["n_grad_steps"])].tobytes(), dtype=GSTEP)
            po = int(h["params_off"])
            self.pleaves = np.frombuffer(buf[po:po + PLEAF.itemsize * int(h["n_param_leaves"])].tobytes(), dtype=PLEAF)
            co = int(h["codes_off"])
            self.codes = np.frombuffer(buf[co:co + int(h["deriv_data_off"]) - co].tobytes(), dtype="u1")
            to = int(h["thetas_off"])
            self.thetas = np.frombuffer(buf[to:to + 8 * int(h["n_params"])].tobytes(), dtype="<f8").copy()
            self.deriv_data = np.zeros_like(self.leaf_data)
            gp, ng = int(h["grad_phases_off"]), int(h["n_grad_phases"])
            self.grad_phases = np.frombuffer(buf[gp:gp + 4 * (ng + 1)].tobytes(), dtype="<u4").astype(np.int64)
            ge = int(h["grad_elem_off_off"])
            self.grad_elem_off = np.frombuffer(buf[ge:ge + 4 * int(h["n_grad_steps"])].tobytes(),
                                               dtype="<u4").astype(np.int64)
            self.gentries = None
            if int(h["gentry_off"]):
                po = int(h["gphase_entry_off"])
                self.gphase_entry = np.frombuffer(buf[po:po + 4 * (ng + 1)].tobytes(), dtype="<u4").astype(np.int64)
                n_ent = int(self.gphase_entry[-1])
                eo = int(h["gentry_off"])
                self.gentries = np.frombuffer(buf[eo:eo + 16 * n_ent].tobytes(), dtype=GENTRY)
                ko = int(h["gktab_off"])
                self.gktab = np.frombuffer(buf[ko:po].tobytes(), dtype="<u4").astype(np.int64)

    def _leaf_reader(self, li, x, o):
        L = self.leaves[li]
        off = int(L["data_off"])
        for f in range(int(L["n_fixed"])):
            src = int(L["fixed_src"][f])
            bit = (x >> src) & 1 if src < 128 else (o >> (src - 128)) & 1
            off += bit << int(L["fixed_pos"][f])
        n = int(L["n_elem"])

        def read(idx):
            assert np.all(idx < n)
            return self.leaf_data[off + idx]
        return read

    def _regtile_step(self, si, A, B, arena):
        """Step si through its register-tiled form: thread t owns the entries
        c0 + c_m[i] + c_n[j]; every entry of C must be owned exactly once."""
        r = self.rtsteps[si]
        st = self.steps[si]
        for f in ("a_off", "b_off", "c_off", "flags", "rc", "nk_ab", "nk_a", "nk_b", "a_cb", "b_cb",
                  "na_runs", "nb_runs"):
            assert int(r[f]) == int(st[f]), f
        rm, rn, nt, rc = int(r["rm"]), int(r["rn"]), int(r["nt"]), int(r["rc"])
        assert 0 < rm + rn and rm <= 3 and rn <= 3 and nt == rc - rm - rn
        t = np.arange(1 << nt, dtype=np.int64)
        c0 = _pext(t, r["free_runs"], int(r["n_free"]))
        ia0 = _pext(c0, r["runs_a"], int(r["na_runs"]))
        ib0 = _pext(c0, r["runs_b"], int(r["nb_runs"]))
        nab, na, nb = int(r["nk_ab"]), int(r["nk_a"]), int(r["nk_b"])
        owned = np.zeros(1 << rc, dtype=np.int64)
        out = {}
        for i in range(1 << rm):
            for j in range(1 << rn):
                c = c0 + int(r["c_m"][i]) + int(r["c_n"][j])
                acc = np.zeros(1 << nt, dtype=np.complex128)
                for k in range(1 << (nab + na + nb)):
                    ka = k & ((1 << (nab + na)) - 1)
                    kb = (k & ((1 << nab) - 1)) | ((k >> (nab + na)) << nab)
                    acc += (A(ia0 + int(r["a_m"][i]) + (ka << int(r["a_cb"]))) *
                            B(ib0 + int(r["b_n"][j]) + (kb << int(r["b_cb"]))))
                np.add.at(owned, c, 1)
                out[(i, j)] = (c, acc)
        assert np.all(owned == 1)
        for c, acc in out.values():
            arena[int(r["c_off"]) + c] = acc

    def _gemm_step(self, si, A, B, arena):
        """Step si through its tensor-core form, as the GEMM kernel defines it: the real
        GEMM [Ar | Ai] x [[Br, Bi], [-Bi, Br]] of three-part bf16 splits (h*h + h*m + m*h +
        h*l + l*h + m*m) accumulated in float64 here. Also checks the kernel's tiling, that
        the GEMM's stores cover C exactly once and that the row operand holds C's unit
        stride."""
        g = self.gemms[si]
        st = self.steps[si]
        nb, nm, nn, nk = (int(g[f]) for f in ("nb", "nm", "nn", "nk"))
        assert nk >= 3 and nm >= 7 and nn >= 3 and int(g["c_off"]) == int(st["c_off"])
        bb, mm, nn_, kk = (np.arange(1 << v, dtype=np.int64) for v in (nb, nm, nn, nk))

        def mv(v, f):
            return _pext(v, g[f], int(g["n_" + f]))
        ia = mv(bb, "ab")[:, None, None] + mv(mm, "am")[None, :, None] + mv(kk, "ak")[None, None, :]
        ib = mv(bb, "bb")[:, None, None] + mv(kk, "bk")[None, :, None] + mv(nn_, "bn")[None, None, :]
        ic = mv(bb, "cb")[:, None, None] + mv(mm, "cm")[None, :, None] + mv(nn_, "cn")[None, None, :]
        assert np.array_equal(np.sort(ic.ravel()), np.arange(1 << int(st["rc"])))
        Ac = np.asarray(A(ia.ravel())).reshape(ia.shape).astype(np.complex64)
        Bc = np.asarray(B(ib.ravel())).reshape(ib.shape).astype(np.complex64)

        def split(v):   # float32 -> three bf16 parts h, m, l (round to nearest even), as float64
            v = np.asarray(v, dtype=np.float32)
            h = _bf16(v)
            r1 = (v - h).astype(np.float32)
            m = _bf16(r1)
            lo = _bf16((r1 - m).astype(np.float32))
            return h.astype(np.float64), m.astype(np.float64), lo.astype(np.float64)
        ar, ai, br, bi = split(Ac.real), split(Ac.imag), split(Bc.real), split(Bc.imag)

        def mm6(x, y):   # h*h + h*m + m*h + h*l + l*h + m*m
            return sum(np.einsum("bmk,bkn->bmn", x[i], y[j]) for i, j in
                       ((0, 0), (0, 1), (1, 0), (0, 2), (2, 0), (1, 1)))
        re = mm6(ar, br) - mm6(ai, bi)
        im = mm6(ai, br) + mm6(ar, bi)
        arena[int(g["c_off"]) + ic] = re + 1j * im
        # C's lowest mode is the row operand's first row mode
        assert any(int(r["src"]) == 0 and int(r["dst"]) == 0 and int(r["len"]) > 0 for r in g["cm"][:int(g["n_cm"])])
        # tiles of the kernel: 128 complex rows, nt real columns (two per complex column, up to
        # 256), chunks of 16 summed entries (8 summed entries fill half of one chunk, the
        # other half holds zeros); the shared-memory core-matrix layout (8-row groups
        # 272 bytes apart, two 128-byte core matrices along the summed index) gives each (row,
        # summed-half) its own 16 bytes
        K, M, N2 = 1 << nk, 1 << nm, 2 << nn
        ntr = 256 if nn >= 7 else N2
        assert (K == 8 or K % 16 == 0) and M % 128 == 0 and N2 % ntr == 0 and ntr in (16, 32, 64, 128, 256)
        for rows in (128, ntr):
            r = np.arange(rows)[:, None]
            half = np.arange(2)[None, :]
            off = (r >> 3) * 272 + half * 128 + (r & 7) * 16
            assert len(np.unique(off)) == off.size and off.max() + 16 <= rows // 8 * 272

    def item_terms(self, x: int, o: int, fused: bool = False, regtile: bool = False, gemm: bool = False):
        """Slice terms of work item (x, o): entry i is slice (o << n_inner) | i. With
        fused=True the steps take their operand offsets from the fused form's tables; with
        regtile=True the steps that have a register-tiled form run through it."""
        h = self.h
        arena = np.zeros(max(int(h["arena_elems"]), 4), dtype=np.complex128)
        for si, st in enumerate(self.steps):
            rc = int(st["rc"])
            c = np.arange(1 << rc, dtype=np.int64)
            flags = int(st["flags"])
            def operand(is_leaf, ref):
                if is_leaf:
                    return self._leaf_reader(int(ref), x, o)
                base = int(ref)

                def read(idx):
                    assert np.all(base + idx < arena.size)
                    return arena[base + idx]
                return read
            A = operand(flags & A_LEAF, st["a_off"])
            unary = flags & UNARY
            B = None if unary else operand(flags & B_LEAF, st["b_off"])
            nab_, na_, nb_ = int(st["nk_ab"]), int(st["nk_a"]), int(st["nk_b"])
            if gemm and self.gemms is not None and int(self.gemms[si]["nk"]) > 0:
                g = self.gemms[si]   # its operands may be the step's in swapped roles
                gf = int(g["flags"])
                self._gemm_step(si, operand(gf & A_LEAF, g["a_off"]), operand(gf & B_LEAF, g["b_off"]), arena)
                continue
            if regtile and int(self.rtsteps[si]["rm"]) + int(self.rtsteps[si]["rn"]) > 0:
                assert not unary
                self._regtile_step(si, A, B, arena)
                continue
            if fused:
                fst = self.fsteps[si]
                for f in ("a_off", "b_off", "c_off", "flags", "rc", "nk_ab", "nk_a", "nk_b", "a_cb", "b_cb"):
                    assert int(fst[f]) == int(st[f]), f
                e = self.tab[int(fst["tab_off"]):int(fst["tab_off"]) + (1 << rc)]
                ia, ib = e & 0xFFFF, (None if unary else e >> 16)
                nk = int(fst["nk"])
                assert nk == nab_ + na_ + nb_
                for k in range(min(1 << nk, 8)):
                    ka = k & ((1 << (nab_ + na_)) - 1)
                    kb = (k & ((1 << nab_) - 1)) | ((k >> (nab_ + na_)) << nab_)
                    assert int(fst["koff_a"][k]) == ka << int(st["a_cb"])
                    assert int(fst["koff_b"][k]) == kb << int(st["b_cb"])
            else:
                ia = _pext(c, st["runs_a"], int(st["na_runs"]))
                ib = None if unary else _pext(c, st["runs_b"], int(st["nb_runs"]))
            nab, na, nb = int(st["nk_ab"]), int(st["nk_a"]), int(st["nk_b"])
            acc = np.zeros(1 << rc, dtype=np.complex128)
            for k in range(1 << (nab + na + nb)):
                ka = k & ((1 << (nab + na)) - 1)
                a = A(ia + (ka << int(st["a_cb"])))
                if unary:
                    acc += a
                else:
                    kb = (k & ((1 << nab) - 1)) | ((k >> (nab + na)) << nab)
                    acc += a * B(ib + (kb << int(st["b_cb"])))
            assert int(st["c_off"]) + (1 << rc) <= arena.size
            arena[int(st["c_off"]):int(st["c_off"]) + (1 << rc)] = acc
        n_in = int(h["n_inner"])
        present = int(h["final_present"])
        n_open, open_present = int(h["n_open"]), int(h["open_present"])
        fin = arena[int(h["final_off"]):]
        scalar = complex(float(h["scalar_re"]), float(h["scalar_im"]))
        zero = (x & (int(h["zero_mask"]) | (int(h["zero_mask_hi"]) << 64))) != 0

        def compress(v, mask, n):
            r, bit = 0, 0
            for j in range(n):
                if (mask >> j) & 1:
                    r |= ((v >> j) & 1) << bit
                    bit += 1
            return r
        out = np.zeros((1 << n_open, 1 << n_in), dtype=np.complex128)
        inner_bits = bin(present).count("1")
        for jo in range(1 << n_open):
            fj = compress(jo, open_present, n_open) << inner_bits
            for i in range(1 << n_in):
                out[jo, i] = 0 if zero else scalar * fin[compress(i, present, n_in) | fj]
        return out if n_open else out[0]

    def slice_terms(self, x: int, fused: bool = False, regtile: bool = False):
        """Slice terms in slice-number order ([2^n_open, slices] with open qubits)."""
        n_out = int(self.h["n_outer"])
        return np.concatenate([self.item_terms(x, o, fused, regtile) for o in range(n_out)], axis=-1)


def _pdep_runs(c, runs, n):
    return _pext(c, runs, n)


def rxy_and_derivative(theta, phi):
    """U = cos(t/2) I - i sin(t/2)(cos(phi) X + sin(phi) Y) and dU/dtheta, [row][column]."""
    c, s = np.cos(theta / 2), np.sin(theta / 2)
    em, ep = np.exp(-1j * phi), np.exp(1j * phi)
    U = np.array([[c, -1j * s * em], [-1j * s * ep, c]])
    dU = np.array([[-s / 2, -0.5j * c * em], [-0.5j * c * ep, -s / 2]])
    return U, dU


def grad_item(prog, x, o, thetas=None, tables=False):
    """(alpha partial, per-slot derivative partials) of work item (x, o) by the image's
    gradient program, with the parametrised leaves rebuilt from `thetas`. tables=True runs
    the per-entry records (GradEntry) phase by phase instead of the gradient steps."""
    h = prog.h
    th = prog.thetas if thetas is None else np.asarray(thetas, dtype=np.float64)
    data = prog.leaf_data.copy()
    deriv = prog.deriv_data.copy()
    for pl in prog.pleaves:
        U, dU = rxy_and_derivative(th[int(pl["param"])], float(pl["phi"]))
        L = prog.leaves[int(pl["leaf"])]
        for e in range(int(pl["n_stored"])):
            code = int(prog.codes[int(pl["code_off"]) + e])
            data[int(L["data_off"]) + e] = U[code >> 1, code & 1]
            deriv[int(L["data_off"]) + e] = dU[code >> 1, code & 1]
    arena = np.zeros(max(int(h["grad_arena_elems"]), 4), dtype=np.complex128)

    def base(L):
        off = int(L["data_off"])
        for f in range(int(L["n_fixed"])):
            src = int(L["fixed_src"][f])
            bit = (x >> src) & 1 if src < 128 else (o >> (src - 128)) & 1
            off += bit << int(L["fixed_pos"][f])
        return off

    def reader(op):
        kind = int(op["kind"])
        if kind == OP_ONE:
            return lambda idx: np.ones(idx.shape, dtype=np.complex128)
        if kind == OP_ARENA:
            b = int(op["off"])
            return lambda idx: arena[b + idx]
        L = prog.leaves[int(op["off"])]
        b = base(L)
        src = data if kind == OP_LEAF else deriv
        return lambda idx: src[b + idx]

    if tables:
        ent = prog.gentries
        meta = ent["meta"].astype(np.int64)
        nk = (meta >> 4) & 15
        srcs = {1: data, 2: deriv}
        for ph in range(len(prog.gphase_entry) - 1):
            e0, e1 = int(prog.gphase_entry[ph]), int(prog.gphase_entry[ph + 1])
            out = np.zeros(e1 - e0, dtype=np.complex128)
            for j in range(e0, e1):
                e = ent[j]
                vals = []
                for kind, r, off in (((meta[j] & 3), int(e["xr"]), int(e["xo"])),
                                     (((meta[j] >> 2) & 3), int(e["yr"]), int(e["yo"]))):
                    vals.append((kind, r, off))

                def val(kind, r, off, dk):
                    if kind == OP_ONE:
                        return 1.0
                    if kind == OP_ARENA:
                        return arena[r + off + dk]
                    return srcs[kind][base(prog.leaves[r]) + off + dk]
                acc = 0j
                for k in range(1 << int(nk[j])):
                    if k == 0:
                        kx = ky = 0
                    else:
                        kp = int(e["k1"]) if nk[j] == 1 else int(prog.gktab[int(e["k1"]) + k - 1])
                        kx, ky = kp & 0xFFFF, kp >> 16
                    acc += val(*vals[0], kx) * val(*vals[1], ky)
                out[j - e0] = acc
            # a phase's records are independent: write after computing all of them
            arena[ent["c"][e0:e1].astype(np.int64)] = out
    for g in ([] if tables else prog.gsteps):
        ro, nk = int(g["ro"]), int(g["nk"])
        oidx = np.arange(1 << ro, dtype=np.int64)
        X, Y = reader(g["x"]), reader(g["y"])
        ox = _pext(oidx, g["x"]["oruns"], int(g["x"]["n_oruns"]))
        oy = _pext(oidx, g["y"]["oruns"], int(g["y"]["n_oruns"]))
        acc = np.zeros(1 << ro, dtype=np.complex128)
        for k in range(1 << nk):
            kk = np.array([k], dtype=np.int64)
            kx = _pext(kk, g["x"]["kruns"], int(g["x"]["n_kruns"]))[0]
            ky = _pext(kk, g["y"]["kruns"], int(g["y"]["n_kruns"]))[0]
            acc += X(ox + kx) * Y(oy + ky)
        arena[int(g["out_off"]):int(g["out_off"]) + (1 << ro)] = acc
    n_in = int(h["n_inner"])
    present = int(h["final_present"])
    fin = arena[int(h["final_fwd_off"]):]
    scalar = complex(float(h["scalar_re"]), float(h["scalar_im"]))
    zero = (x & (int(h["zero_mask"]) | (int(h["zero_mask_hi"]) << 64))) != 0
    tot = 0j
    for i in range(1 << n_in):
        fi, bit = 0, 0
        for j in range(n_in):
            if (present >> j) & 1:
                fi |= ((i >> j) & 1) << bit
                bit += 1
        tot += fin[fi]
    npl = int(h["n_param_leaves"])
    slots = arena[int(h["gslot_off"]):int(h["gslot_off"]) + npl] * scalar
    if zero:
        return 0j, np.zeros(npl, dtype=np.complex128)
    return scalar * tot, slots


def grad(prog, x, thetas=None, tables=False):
    """(alpha, d alpha / d theta per parameter) over every work item."""
    n_out = int(prog.h["n_outer"])
    a = 0j
    slots = np.zeros(int(prog.h["n_param_leaves"]), dtype=np.complex128)
    for o in range(n_out):
        ai, si = grad_item(prog, x, o, thetas, tables)
        a += ai
        slots += si
    g = np.zeros(int(prog.h["n_params"]), dtype=np.complex128)
    for i, pl in enumerate(prog.pleaves):
        g[int(pl["param"])] += slots[i]
    return a, g


def check_schedule(prog):
    """The fused phases: every step in exactly one phase, each phase's steps independent
    (no step reads another's output of the same phase, no output overlaps an operand or
    output of its phase), each step's lanes contiguous and numbered 0..count-1."""
    lanes = int(prog.h["fused_lanes"])
    seen = {}
    for ph, row in enumerate(prog.lane_map):
        steps = {}
        for lane, m in enumerate(row):
            if m == 0xFFFFFFFF:
                continue
            s, sub, cnt = int(m) & 0xFFF, (int(m) >> 12) & 0x3FF, int(m) >> 22
            steps.setdefault(s, []).append((lane, sub, cnt))
        for s, ls in steps.items():
            assert s not in seen
            seen[s] = ph
            cnt = ls[0][2]
            assert [x[1] for x in ls] == list(range(cnt)) and all(x[2] == cnt for x in ls)
            assert [x[0] for x in ls] == list(range(ls[0][0], ls[0][0] + cnt))
        ranges = []
        for s in steps:
            st = prog.steps[s]
            out = (int(st["c_off"]), int(st["c_off"]) + (1 << int(st["rc"])))
            ins = []
            for fl, key in ((2, "a_off"), (4, "b_off")):
                if fl == 4 and int(st["flags"]) & 1:
                    continue
                if not int(st["flags"]) & fl:
                    ins.append(int(st[key]))
            ranges.append((out, ins))
        for i, (out_i, _) in enumerate(ranges):
            for j, (out_j, ins_j) in enumerate(ranges):
                if i == j:
                    continue
                assert out_i[1] <= out_j[0] or out_j[1] <= out_i[0]       # outputs disjoint
                for a in ins_j:
                    assert not (out_i[0] <= a < out_i[1])                  # no read of a same-phase output
    assert sorted(seen) == list(range(len(prog.steps)))
    assert lanes % 32 == 0


def check_grad_schedule(prog):
    """Gradient phases cover the steps in order; entry offsets are each phase's prefix sums;
    no step reads an arena range written by another step of its phase."""
    ph = prog.grad_phases
    assert ph[0] == 0 and ph[-1] == len(prog.gsteps) and np.all(np.diff(ph) > 0)
    for i in range(len(ph) - 1):
        acc, outs, reads = 0, [], []
        for g in range(ph[i], ph[i + 1]):
            st = prog.gsteps[g]
            assert prog.grad_elem_off[g] == acc
            acc += 1 << int(st["ro"])
            o0 = int(st["out_off"])
            outs.append((o0, o0 + (1 << int(st["ro"]))))
            for op in (st["x"], st["y"]):
                if int(op["kind"]) != OP_ARENA:
                    continue
                hi = _pext(np.array([(1 << int(st["ro"])) - 1]), op["oruns"], int(op["n_oruns"]))[0] + \
                    _pext(np.array([(1 << int(st["nk"])) - 1]), op["kruns"], int(op["n_kruns"]))[0]
                reads.append((int(op["off"]), int(op["off"]) + int(hi) + 1))
        for a0, a1 in outs:
            for b0, b1 in reads:
                assert a1 <= b0 or b1 <= a0, "a step reads another step's output in the same phase"
        outs.sort()
        for (a0, a1), (b0, b1) in zip(outs, outs[1:]):
            assert a1 <= b0
