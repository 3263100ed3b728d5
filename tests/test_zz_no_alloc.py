"""gbr_crt_noalloc: Chinese remaindering without any allocation.

Callers that may not allocate device memory when they need a result (a host
that fixes its GPU memory up front, code inside another framework's allocator
or memory pool, loops that cannot take the synchronisation cudaMalloc may
bring) reconstruct integers with gbr_crt_noalloc, which works only in the
buffers they pass plus the library's fixed device array.  This test feeds it
the residues of resultants that the ordinary entry point computed and checks
that it rebuilds exactly those resultants, on two calls in a row (the fixed
array keeps the first call's digits when the second starts).
"""

import ctypes as C

import numpy as np
import pytest

from paper_1103_4697_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _noalloc(values, k, limbs, pad=0):
    """Residues of `values` modulo the first k table primes -> gbr_crt_noalloc -> ints
    (rows of the residue array `pad` words longer than the coefficient count)."""
    import torch

    from paper_1103_4697_gb300 import native as N
    from paper_1103_4697_gb300.api import primes

    ps = primes(k)
    n = len(values)
    stride = n + pad
    res = np.zeros((k, stride), dtype=np.uint32)
    for i, p in enumerate(ps):
        res[i, :n] = [v % p for v in values]
        res[i, n:] = 0xFFFFFFFF                      # not a residue: must never be read
    d_res = torch.from_numpy(res.reshape(-1).view(np.int32)).cuda()
    d_mag = torch.full((n * limbs,), -1, dtype=torch.int32, device="cuda")   # stale contents on purpose
    d_sign = torch.full((n,), 7, dtype=torch.int8, device="cuda")
    stream = torch.cuda.current_stream()
    st = N.lib().gbr_crt_noalloc(C.c_void_p(d_res.data_ptr()), k, n, stride, C.c_void_p(d_mag.data_ptr()), limbs,
                                 C.c_void_p(d_sign.data_ptr()), C.c_void_p(stream.cuda_stream))
    assert st == N.OK
    stream.synchronize()
    mag = d_mag.cpu().numpy().view(np.uint32).reshape(n, limbs)
    sgn = d_sign.cpu().numpy()
    out = []
    for c in range(n):
        v = int.from_bytes(mag[c].astype("<u4").tobytes(), "little")
        out.append(-v if sgn[c] < 0 else v)
    return out


def test_noalloc_crt_matches_resultant_entry_point():
    from paper_1103_4697_gb300.api import Context, resultant_info

    f, g = W.deg20_pair(2)
    with Context(device=0, mem_budget=1 << 30) as ctx:
        r1 = ctx.resultant(f, g)
        r2 = ctx.discriminant_res(f)
    i1 = resultant_info(f, g)
    i2 = resultant_info(f, None, disc=True)
    # two calls in a row on the same stream; the second sees the first's digits
    assert _noalloc(r1, i1["primes"], i1["limbs"]) == r1
    assert _noalloc(r2, i2["primes"], i2["limbs"]) == r2


def test_noalloc_crt_at_its_limits():
    """k = 64 primes and 16 384 coefficients fill the fixed array exactly; the row
    stride is above the coefficient count; values include the ends of the symmetric
    range (0, +-1, +-(M-1)/2, where the digit comparison and the +1 carry of negative
    values decide), checked against Python integers on two calls in a row."""
    import random

    from paper_1103_4697_gb300.api import primes

    k, n = 64, 16384
    M = 1
    for p in primes(k):
        M *= p
    h = (M - 1) // 2
    rng = random.Random(64)
    edge = [0, 1, -1, h, -h, h - 1, -(h - 1), 2, -2]
    vals = edge + [rng.randrange(-h, h + 1) for _ in range(n - len(edge) - 64)]
    vals += [rng.randrange(-2 ** rng.randrange(1, 1900), 2 ** rng.randrange(1, 1900)) for _ in range(64)]
    assert len(vals) == n and all(-h <= v <= h for v in vals)
    limbs = 64
    assert _noalloc(vals, k, limbs, pad=37) == vals
    rev = vals[::-1]
    assert _noalloc(rev, k, limbs, pad=5) == rev


def test_noalloc_rejects_sizes_beyond_its_array():
    from paper_1103_4697_gb300 import native as N

    L = N.lib()
    dummy = C.c_void_p(1)
    assert L.gbr_crt_noalloc(dummy, 65, 10, 10, dummy, 100, dummy, None) == N.ELIMIT
    assert L.gbr_crt_noalloc(dummy, 64, 20000, 20000, dummy, 64, dummy, None) == N.ELIMIT
    assert L.gbr_crt_noalloc(dummy, 8, 10, 10, dummy, 2, dummy, None) == N.EINVAL
