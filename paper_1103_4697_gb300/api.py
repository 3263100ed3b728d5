"""Python binding of libgbres: argument marshalling only.

Every step of the resultant and gcd path runs in the library's CUDA kernels;
this module converts numpy arrays / Python ints to the C structures of
include/gbres.h and the sign-magnitude results back to Python ints.  PyTorch
supplies the device workspace (a uint8 tensor the context sub-allocates from)
and the stream.

Polynomial conventions: a bivariate polynomial is a 2-D array ``f[j][i]`` =
coefficient of x^i y^j (numpy int64, or any nested sequence of Python ints of
any size); a univariate polynomial is a 1-D sequence ``p[i]`` = coefficient of
x^i.  Results are lists of Python ints, lowest power first, with no trailing
zeros (the zero polynomial is ``[]``).
"""

from __future__ import annotations

import ctypes as C

import numpy as np

from . import native as N

_BIPOLY_DT = np.dtype([("deg_x", np.int32), ("deg_y", np.int32), ("words", np.int32), ("pad", np.int32),
                       ("coef", np.uint64)])
_UPOLY_DT = np.dtype([("deg", np.int32), ("words", np.int32), ("coef", np.uint64)])
assert _BIPOLY_DT.itemsize == C.sizeof(N.BiPoly) and _UPOLY_DT.itemsize == C.sizeof(N.UPoly)

_M64 = (1 << 64) - 1


def _words_for(vals) -> int:
    b = max((int(v).bit_length() for v in vals), default=0)
    return max(1, (b + 1 + 63) // 64)


def _to_words(arr, W: int) -> np.ndarray:
    """Flattened two's-complement words of the integers in `arr` (row-major)."""
    flat = np.asarray(arr, dtype=object).ravel() if not (isinstance(arr, np.ndarray) and arr.dtype == np.int64) \
        else arr.ravel()
    if W == 1:
        return np.asarray(flat, dtype=np.int64).view(np.uint64)
    # each value's two's complement in W words, least significant first
    mask = (1 << (64 * W)) - 1
    raw = b"".join((int(v) & mask).to_bytes(8 * W, "little") for v in flat)
    return np.frombuffer(raw, dtype="<u8").astype(np.uint64)


def _as_2d(f):
    if isinstance(f, np.ndarray) and f.ndim == 2:
        return f
    rows = [[int(c) for c in r] for r in f]
    width = max((len(r) for r in rows), default=1) or 1
    padded = [r + [0] * (width - len(r)) for r in rows] or [[0] * width]
    try:
        return np.array(padded, dtype=np.int64)    # every coefficient fits a signed word
    except OverflowError:
        a = np.empty((len(padded), width), dtype=object)
        a[:, :] = padded
        return a


class _Packed:
    """Keeps the coefficient words alive while the C call runs."""

    def __init__(self):
        self.bufs = []


def pack_bipolys(polys, keep: _Packed):
    """Array of gbr_bipoly for a list of 2-D arrays or a 3-D int64 array."""
    if isinstance(polys, np.ndarray) and polys.ndim == 3 and polys.dtype == np.int64:
        arr = np.ascontiguousarray(polys)
        keep.bufs.append(arr)
        n, ry, rx = arr.shape
        desc = np.zeros(n, dtype=_BIPOLY_DT)
        desc["deg_x"] = rx - 1
        desc["deg_y"] = ry - 1
        desc["words"] = 1
        desc["coef"] = arr.ctypes.data + np.arange(n, dtype=np.uint64) * np.uint64(ry * rx * 8)
        keep.bufs.append(desc)
        return desc
    desc = np.zeros(len(polys), dtype=_BIPOLY_DT)
    for k, f in enumerate(polys):
        a = _as_2d(f)
        W = 1 if a.dtype == np.int64 else _words_for(a.ravel())
        w = np.ascontiguousarray(_to_words(a, W))
        keep.bufs.append(w)
        desc[k] = (a.shape[1] - 1, a.shape[0] - 1, W, 0, w.ctypes.data)
    keep.bufs.append(desc)
    return desc


def pack_upolys(polys, keep: _Packed):
    desc = np.zeros(len(polys), dtype=_UPOLY_DT)
    # int64 coefficients: one contiguous buffer, filled by numpy
    try:
        lens = np.array([max(len(p), 1) for p in polys], dtype=np.int64)
        offs = np.zeros(len(polys), dtype=np.int64)
        if len(polys):
            offs[1:] = np.cumsum(lens)[:-1]
        flat = np.zeros(int(lens.sum()) if len(polys) else 1, dtype=np.int64)
        for p, o in zip(polys, offs):
            if len(p):
                flat[o:o + len(p)] = p
        keep.bufs.append(flat)
        desc["deg"] = lens - 1
        desc["words"] = 1
        desc["coef"] = flat.ctypes.data + 8 * offs
        keep.bufs.append(desc)
        return desc
    except OverflowError:
        pass
    for k, p in enumerate(polys):
        vals = [int(c) for c in p] or [0]
        W = _words_for(vals)
        w = np.ascontiguousarray(_to_words(np.array(vals, dtype=object), W))
        keep.bufs.append(w)
        desc[k] = (len(vals) - 1, W, w.ctypes.data)
    keep.bufs.append(desc)
    return desc


def bigpoly_to_ints(b: N.BigPoly) -> list[int]:
    if b.deg < 0:
        return []
    n, L = b.deg + 1, b.limbs
    mag = np.ctypeslib.as_array(b.mag, shape=(n * L,)).reshape(n, L)
    sgn = np.ctypeslib.as_array(b.sign, shape=(n,))
    raw = memoryview(mag.astype("<u4").tobytes())   # slices of a memoryview are not copies
    step = 4 * L
    out = [int.from_bytes(raw[i * step:(i + 1) * step], "little") for i in range(n)]
    for i, sg in enumerate(sgn.tolist()):
        if sg < 0:
            out[i] = -out[i]
    while out and out[-1] == 0:
        out.pop()
    return out


def pack_bigpolys(polys, keep: _Packed):
    """Integer polynomials (ascending coefficients) in the gbr_bigpoly layout:
    little-endian 32-bit limbs of |c| and a sign byte per coefficient."""
    arr = (N.BigPoly * max(len(polys), 1))()
    for k, p in enumerate(polys):
        vals = [int(c) for c in p]
        while vals and vals[-1] == 0:
            vals.pop()
        if not vals:
            arr[k].deg, arr[k].limbs = -1, 1
            continue
        L = max(1, max((abs(v).bit_length() + 31) // 32 for v in vals))
        raw = b"".join(abs(v).to_bytes(4 * L, "little") for v in vals)
        mag = np.frombuffer(raw, dtype="<u4").copy()
        sgn = np.array([(v > 0) - (v < 0) for v in vals], dtype=np.int8)
        keep.bufs += [mag, sgn]
        arr[k].deg, arr[k].limbs = len(vals) - 1, L
        arr[k].mag = mag.ctypes.data_as(C.POINTER(C.c_uint32))
        arr[k].sign = sgn.ctypes.data_as(C.POINTER(C.c_int8))
    keep.bufs.append(arr)
    return arr


def _ptr(desc) -> C.c_void_p:
    return C.c_void_p(desc.ctypes.data)


class Resident:
    """Inputs uploaded once to device memory (gbr_upload_pairs)."""

    def __init__(self, ctx: "Context", handle: C.c_void_p, n: int):
        self.ctx, self.handle, self.n = ctx, handle, n

    def run(self):
        N.check(N.lib().gbr_run_resident(self.ctx.handle, self.handle), self.ctx.handle)

    def fetch(self, first: int = 0, count: int | None = None) -> list[list[int]]:
        count = self.n - first if count is None else count
        outs = (N.BigPoly * max(count, 1))()
        N.check(N.lib().gbr_fetch_resident(self.ctx.handle, self.handle, first, count, outs), self.ctx.handle)
        return self.ctx._collect(outs, count)

    def plan(self, first: int = 0, count: int | None = None) -> list[dict]:
        """gbr_resident_plan: the device's plan per job after a run (degrees, the degree
        bound of the result, primes, limbs, log2 of the coefficient bound)."""
        count = self.n - first if count is None else count
        outs = (N.ResInfo * max(count, 1))()
        N.check(N.lib().gbr_resident_plan(self.ctx.handle, self.handle, first, count, outs), self.ctx.handle)
        return [{k: getattr(outs[i], k) for k, _ in N.ResInfo._fields_} for i in range(count)]

    def free(self):
        if self.handle:
            N.lib().gbr_free_resident(self.ctx.handle, self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Context:
    """A libgbres context on one CUDA device, with a torch-allocated workspace."""

    def __init__(self, device: int = 0, mem_budget: int = 4 << 30, stream=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("libgbres needs a CUDA device; there is no CPU fallback")
        L = N.lib()
        self.device = device
        torch.cuda.set_device(device)
        self.workspace = torch.empty(int(mem_budget), dtype=torch.uint8, device=f"cuda:{device}")
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        h = C.c_void_p()
        N.check(L.gbr_create(C.byref(h), device, int(mem_budget), C.c_void_p(self.workspace.data_ptr()),
                             C.c_void_p(self.stream.cuda_stream)))
        self.handle = h

    # ------------------------------------------------------------- lifecycle
    def close(self):
        if getattr(self, "handle", None):
            N.lib().gbr_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------- helpers
    def _collect(self, outs, count: int) -> list[list[int]]:
        L = N.lib()
        res = []
        for i in range(count):
            res.append(bigpoly_to_ints(outs[i]))
            L.gbr_free_result(self.handle, C.byref(outs[i]))
        return res

    def set_option(self, opt: int, value: int):
        N.check(N.lib().gbr_set_option(self.handle, opt, int(value)), self.handle)

    def calibrate(self) -> dict:
        """Measured Montgomery multiply and fused multiply-subtract rates of this GPU."""
        cal = N.Calib()
        N.check(N.lib().gbr_calibrate(self.handle, C.byref(cal)), self.handle)
        return {k: getattr(cal, k) for k, _ in N.Calib._fields_}

    def stats(self) -> dict:
        s = N.Stats()
        N.check(N.lib().gbr_get_stats(self.handle, C.byref(s)), self.handle)
        return {k: getattr(s, k) for k, _ in N.Stats._fields_}

    # ------------------------------------------------------------- resultants
    def resultant_batch(self, fs, gs, var: int = 1) -> list[list[int]]:
        keep = _Packed()
        df, dg = pack_bipolys(fs, keep), pack_bipolys(gs, keep)
        n = len(df)
        outs = (N.BigPoly * max(n, 1))()
        N.check(N.lib().gbr_resultant_batch(self.handle, n, _ptr(df), _ptr(dg), var, outs), self.handle)
        return self._collect(outs, n)

    def discriminant_res_batch(self, fs, var: int = 1) -> list[list[int]]:
        keep = _Packed()
        df = pack_bipolys(fs, keep)
        n = len(df)
        outs = (N.BigPoly * max(n, 1))()
        N.check(N.lib().gbr_discriminant_res_batch(self.handle, n, _ptr(df), var, outs), self.handle)
        return self._collect(outs, n)

    def resultant(self, f, g, var: int = 1) -> list[int]:
        keep = _Packed()
        df, dg = pack_bipolys([f], keep), pack_bipolys([g], keep)
        out = N.BigPoly()
        N.check(N.lib().gbr_resultant(self.handle, C.cast(_ptr(df), C.POINTER(N.BiPoly)),
                                      C.cast(_ptr(dg), C.POINTER(N.BiPoly)), var, C.byref(out)), self.handle)
        r = bigpoly_to_ints(out)
        N.lib().gbr_free_result(self.handle, C.byref(out))
        return r

    def discriminant_res(self, f, var: int = 1) -> list[int]:
        keep = _Packed()
        df = pack_bipolys([f], keep)
        out = N.BigPoly()
        N.check(N.lib().gbr_discriminant_res(self.handle, C.cast(_ptr(df), C.POINTER(N.BiPoly)), var,
                                             C.byref(out)), self.handle)
        r = bigpoly_to_ints(out)
        N.lib().gbr_free_result(self.handle, C.byref(out))
        return r

    def upload_pairs(self, fs, gs=None, var: int = 1, disc: bool = False) -> Resident:
        keep = _Packed()
        df = pack_bipolys(fs, keep)
        dg = pack_bipolys(gs, keep) if gs is not None else None
        h = C.c_void_p()
        N.check(N.lib().gbr_upload_pairs(self.handle, len(df), _ptr(df), _ptr(dg) if dg is not None else None,
                                         var, int(disc), C.byref(h)), self.handle)
        return Resident(self, h, len(df))

    # ------------------------------------------------------------- arrangements
    def arrangement_resultants(self, fs, var: int = 1) -> tuple[list[list[int]], dict]:
        """gbr_arrangement_resultants: ([res(f_i, d f_i/dvar) for i], {(i, j): res(f_i, f_j)
        for i < j}) for the curves fs (Section 3, curve-pair analysis)."""
        keep = _Packed()
        df = pack_bipolys(fs, keep)
        n = len(df)
        nj = n * (n + 1) // 2
        outs = (N.BigPoly * max(nj, 1))()
        N.check(N.lib().gbr_arrangement_resultants(self.handle, n, _ptr(df), var, outs), self.handle)
        res = self._collect(outs, nj)
        pairs, q = {}, n
        for i in range(n):
            for j in range(i + 1, n):
                pairs[(i, j)] = res[q]
                q += 1
        return res[:n], pairs

    def upload_arrangement(self, fs, var: int = 1) -> Resident:
        """gbr_upload_arrangement: a resident batch of the n(n + 1)/2 arrangement jobs
        (the n discriminant-type resultants first, then the pairs in row-major order)."""
        keep = _Packed()
        df = pack_bipolys(fs, keep)
        h = C.c_void_p()
        N.check(N.lib().gbr_upload_arrangement(self.handle, len(df), _ptr(df), var, C.byref(h)), self.handle)
        n = len(df)
        return Resident(self, h, n * (n + 1) // 2)

    # ------------------------------------------------------------- gcd
    def gcd_batch(self, ps, qs) -> list[list[int]]:
        keep = _Packed()
        dp, dq = pack_upolys(ps, keep), pack_upolys(qs, keep)
        n = len(dp)
        outs = (N.BigPoly * max(n, 1))()
        N.check(N.lib().gbr_gcd_batch(self.handle, n, _ptr(dp), _ptr(dq), outs), self.handle)
        return self._collect(outs, n)

    def mixed_batch(self, fs, gs, ps, qs, var: int = 1) -> tuple[list[list[int]], list[list[int]]]:
        """gbr_mixed_batch: res_var(fs[i], gs[i]) and gcd(ps[j], qs[j]) in one call."""
        keep = _Packed()
        df, dg = pack_bipolys(fs, keep), pack_bipolys(gs, keep)
        dp, dq = pack_upolys(ps, keep), pack_upolys(qs, keep)
        nr, ng = len(df), len(dp)
        ro, go = (N.BigPoly * max(nr, 1))(), (N.BigPoly * max(ng, 1))()
        N.check(N.lib().gbr_mixed_batch(self.handle, nr, _ptr(df), _ptr(dg), var, ro, ng, _ptr(dp), _ptr(dq), go),
                self.handle)
        return self._collect(ro, nr), self._collect(go, ng)

    def gcd(self, p, q) -> list[int]:
        return self.gcd_batch([p], [q])[0]

    # ------------------------------------------------------------- gcd with cofactors, bivariate gcd
    def gcd_cofactors_batch(self, ps, qs) -> list[tuple[list[int], list[int], list[int]]]:
        """gbr_gcd_cofactors_batch: (gcd, p / gcd, q / gcd) per pair."""
        keep = _Packed()
        dp, dq = pack_upolys(ps, keep), pack_upolys(qs, keep)
        n = len(dp)
        g, a, b = ((N.BigPoly * max(n, 1))() for _ in range(3))
        N.check(N.lib().gbr_gcd_cofactors_batch(self.handle, n, _ptr(dp), _ptr(dq), g, a, b), self.handle)
        return list(zip(self._collect(g, n), self._collect(a, n), self._collect(b, n)))

    def _bigbipoly_rows(self, x) -> list[list[int]]:
        if x.deg_y < 0:
            out = []
        else:
            flat = bigpoly_to_ints(N.BigPoly(x.c.deg, x.c.limbs, x.c.mag, x.c.sign))
            w = x.deg_x + 1
            flat = flat + [0] * ((x.deg_y + 1) * w - len(flat))
            out = [flat[j * w:(j + 1) * w] for j in range(x.deg_y + 1)]
        N.lib().gbr_free_bigbipoly(self.handle, C.byref(x))
        return out

    def gcd2_batch(self, fs, gs):
        """gbr_gcd2_batch: (h, f / h, g / h) per pair, each as rows (row j = coefficients
        of y^j, lowest power of x first; [] for zero)."""
        keep = _Packed()
        df, dg = pack_bipolys(fs, keep), pack_bipolys(gs, keep)
        n = len(df)
        h, a, b = ((N.BigBiPoly * max(n, 1))() for _ in range(3))
        N.check(N.lib().gbr_gcd2_batch(self.handle, n, _ptr(df), _ptr(dg), h, a, b), self.handle)
        return [(self._bigbipoly_rows(h[i]), self._bigbipoly_rows(a[i]), self._bigbipoly_rows(b[i])) for i in range(n)]

    def content_batch(self, fs, var: int = 1) -> list[list[int]]:
        """gbr_content_batch: the content of each curve with respect to var (Section 2,
        content removal), a polynomial in the other variable."""
        keep = _Packed()
        df = pack_bipolys(fs, keep)
        n = len(df)
        outs = (N.BigPoly * max(n, 1))()
        N.check(N.lib().gbr_content_batch(self.handle, n, _ptr(df), var, outs), self.handle)
        return self._collect(outs, n)

    def teissier_res_batch(self, fs) -> list[list[int]]:
        """gbr_teissier_res_batch: Q = res(f_x / h, f_y / h, y), h = gcd(f_x, f_y)
        (Section 2.1)."""
        keep = _Packed()
        df = pack_bipolys(fs, keep)
        n = len(df)
        outs = (N.BigPoly * max(n, 1))()
        N.check(N.lib().gbr_teissier_res_batch(self.handle, n, _ptr(df), outs), self.handle)
        return self._collect(outs, n)

    # ------------------------------------------------------------- square-free factorisation
    def squarefree_batch(self, rs) -> list[tuple[int, list[list[int]]]]:
        """gbr_squarefree_batch: for each R, (u, [r_1, ..., r_m]) with
        R = u * prod r_i^i (Section 2.1), every r_i primitive with a positive
        leading coefficient; R = 0 gives (0, [])."""
        keep = _Packed()
        arr = pack_bigpolys(rs, keep)
        n = len(rs)
        outs = (N.Sqf * max(n, 1))()
        L = N.lib()
        N.check(L.gbr_squarefree_batch(self.handle, n, arr, outs), self.handle)
        res = []
        for i in range(n):
            u = bigpoly_to_ints(outs[i].unit)
            facs = [bigpoly_to_ints(outs[i].factors[k]) for k in range(outs[i].count)]
            L.gbr_free_sqf(self.handle, C.byref(outs[i]))
            res.append((u[0] if u else 0, [f if f else [0] for f in facs]))
        return res

    def squarefree(self, r) -> tuple[int, list[list[int]]]:
        return self.squarefree_batch([r])[0]


def resultant_info(f, g=None, var: int = 1, disc: bool = False) -> dict:
    """Host-side plan of one resultant (degrees, bound, primes); needs no device."""
    keep = _Packed()
    df = pack_bipolys([f], keep)
    dg = pack_bipolys([g if g is not None else [[0]]], keep)
    info = N.ResInfo()
    N.check(N.lib().gbr_resultant_info(C.cast(_ptr(df), C.POINTER(N.BiPoly)), C.cast(_ptr(dg), C.POINTER(N.BiPoly)),
                                       var, int(disc), C.byref(info)))
    return {k: getattr(info, k) for k, _ in N.ResInfo._fields_}


def primes(k: int) -> list[int]:
    """The first k primes of the library's fixed table (host only)."""
    L = N.lib()
    out = []
    for i in range(k):
        p = C.c_uint32()
        N.check(L.gbr_prime(i, C.byref(p)))
        out.append(p.value)
    return out


def _job(kind: int, a, b, var: int, keep: _Packed) -> N.Job:
    j = N.Job()
    j.kind, j.var = kind, var
    if kind == N.JOB_GCD:
        d = pack_upolys([a, b], keep)
        j.p = N.UPoly(int(d[0]["deg"]), int(d[0]["words"]), int(d[0]["coef"]))
        j.q = N.UPoly(int(d[1]["deg"]), int(d[1]["words"]), int(d[1]["coef"]))
    else:
        polys = [a, b] if kind == N.JOB_RESULTANT else [a, a]
        d = pack_bipolys(polys, keep)
        j.f = N.BiPoly(int(d[0]["deg_x"]), int(d[0]["deg_y"]), int(d[0]["words"]), int(d[0]["coef"]))
        j.g = N.BiPoly(int(d[1]["deg_x"]), int(d[1]["deg_y"]), int(d[1]["words"]), int(d[1]["coef"]))
    return j


def _submit(self, kind: int, a, b=None, var: int = 1) -> int:
    """gbr_submit: queue a resultant (kind JOB_RESULTANT), res(f, f') (JOB_DISC) or gcd
    (JOB_GCD) job; returns its ticket.  The job's data is copied by the library."""
    keep = _Packed()
    j = _job(kind, a, b, var, keep)
    t = C.c_uint64()
    N.check(N.lib().gbr_submit(self.handle, C.byref(j), C.byref(t)), self.handle)
    return t.value


def _poll(self, ticket: int, timeout_ms: int = -1):
    """gbr_poll: the job's result as a list of ints, or None if not finished in time."""
    out = N.BigPoly()
    st = N.lib().gbr_poll(self.handle, C.c_uint64(ticket), C.byref(out), int(timeout_ms))
    if st in (N.EAGAIN, N.ETIMEOUT):
        return None
    N.check(st, self.handle)
    r = bigpoly_to_ints(out)
    N.lib().gbr_free_result(self.handle, C.byref(out))
    return r


def _wait_any(self, timeout_ms: int = -1):
    """gbr_wait_any: (ticket, result as a list of ints, completion time in seconds on
    gbr_clock) of the next finished job, or None when none finished in time or no
    job is outstanding."""
    out = N.BigPoly()
    t = C.c_uint64()
    td = C.c_double()
    st = N.lib().gbr_wait_any(self.handle, int(timeout_ms), C.byref(t), C.byref(out), C.byref(td))
    if st in (N.EAGAIN, N.ETIMEOUT, N.ENOTFOUND):
        return None
    N.check(st, self.handle)
    r = bigpoly_to_ints(out)
    N.lib().gbr_free_result(self.handle, C.byref(out))
    return t.value, r, td.value


def _serve_stats(self) -> dict:
    s = N.ServeStats()
    N.check(N.lib().gbr_get_serve_stats(self.handle, C.byref(s)), self.handle)
    return {k: getattr(s, k) for k, _ in N.ServeStats._fields_}


Context.submit = _submit
Context.poll = _poll
Context.wait_any = _wait_any
Context.serve_stats = _serve_stats
