"""The allocation-free entry point ejoin_threshold_static.

It exists for callers that cannot call cudaMalloc (a pool-owning database
executor or server, a fixed memory budget, a latency-critical loop where an
allocation would synchronise the device).  These tests call it through the C
ABI: twice in a row, on different inputs, against the context-based
ejoin_threshold (BF16) on the same inputs (the same pair set, similarities
within 1e-5); on a small join against the FP64 oracle (the parity rule of
the other GPU tests); and in both overflow cases the header documents.  The
file is collected last so that a run that stops at the first failure has run
every other test first; it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import oracle
from parity_util import compare

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2312_01476_gb300 as pkg  # noqa: E402
from paper_2312_01476_gb300 import ejoin as E  # noqa: E402


def _lib():
    lib = E.load_library()
    lib.ejoin_threshold_static.restype = ctypes.c_int
    lib.ejoin_threshold_static.argtypes = [E.ejoin_rel, E.ejoin_rel, ctypes.c_float, ctypes.c_void_p,
                                           ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64), ctypes.c_void_p]
    return lib


def _static_join(lib, R, S, eps, capacity):
    out = torch.empty((capacity, 3), dtype=torch.int32, device="cuda")
    cnt = ctypes.c_uint64(0)
    st = lib.ejoin_threshold_static(E._dev_rel(R), E._dev_rel(S), ctypes.c_float(eps),
                                    ctypes.c_void_p(out.data_ptr()), capacity, ctypes.byref(cnt),
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, int(cnt.value), out


def _as_dict(i, j, s):
    return dict(zip(zip(i.tolist(), j.tolist()), s.tolist()))


def test_static_matches_context_path_on_two_calls():
    lib = _lib()
    cases = [(3000, 1700, 300, 0.15, 11), (700, 4100, 128, 0.2, 12)]
    for nR, nS, d, eps, seed in cases:
        rng = np.random.default_rng(seed)
        R = torch.from_numpy(rng.standard_normal((nR, d)).astype(np.float32)).cuda()
        S = torch.from_numpy(rng.standard_normal((nS, d)).astype(np.float32)).cuda()
        with pkg.Ctx(device=0, prec="bf16") as ctx:
            ref = pkg.ejoin_threshold(ctx, R, S, eps)
            want = _as_dict(ref.i.cpu().numpy(), ref.j.cpu().numpy(), ref.sim.cpu().numpy())
        assert len(want) > 1000
        st, n, out = _static_join(lib, R, S, eps, len(want) + 4096)
        assert st == 0, pkg.ejoin_strerror(st)
        assert n == len(want)
        o = out[:n].cpu().numpy()
        got = _as_dict(o[:, 0], o[:, 1], o[:, 2].view(np.float32))
        assert set(got) == set(want)
        err = max(abs(got[k] - want[k]) for k in want)
        assert err <= 1e-5


def test_static_rejects_sizes_beyond_the_limit():
    lib = _lib()
    big = torch.empty((70000, 8), dtype=torch.float32, device="cuda")
    small = torch.zeros((10, 8), dtype=torch.float32, device="cuda")
    st, n, _ = _static_join(lib, big, small, 0.5, 16)
    assert st == E.EJOIN_EINVAL and n == 0
    wide = torch.empty((40000, 512), dtype=torch.float32, device="cuda")
    st, n, _ = _static_join(lib, wide, small.new_zeros((10, 512)), 0.5, 16)
    assert st == E.EJOIN_EINVAL


def test_static_matches_the_oracle():
    lib = _lib()
    rng = np.random.default_rng(21)
    centres = rng.standard_normal((12, 64))
    Rn = (centres[rng.integers(0, 12, 300)] + 0.5 * rng.standard_normal((300, 64)) / 8).astype(np.float32)
    Sn = (centres[rng.integers(0, 12, 200)] + 0.5 * rng.standard_normal((200, 64)) / 8).astype(np.float32)
    eps = 0.9
    oi, oj, os_ = oracle.join(Rn, Sn, eps)
    assert len(oi) > 500
    st, n, out = _static_join(lib, torch.from_numpy(Rn).cuda(), torch.from_numpy(Sn).cuda(), eps, len(oi) + 4096)
    assert st == 0, pkg.ejoin_strerror(st)
    o = out[:n].cpu().numpy()
    compare(Rn, Sn, eps, o[:, 0].view(np.uint32), o[:, 1].view(np.uint32), o[:, 2].view(np.float32), oi, oj, os_)


def test_static_overflow_cases():
    lib = _lib()
    rng = np.random.default_rng(22)
    R = torch.from_numpy(rng.standard_normal((1100, 32)).astype(np.float32)).cuda()
    S = torch.from_numpy(rng.standard_normal((1000, 32)).astype(np.float32)).cuda()
    # more result pairs than the caller's capacity: the exact count, the first `capacity` records valid
    eps = 0.3
    st, n_full, full = _static_join(lib, R, S, eps, 1 << 18)
    assert st == 0 and 1000 < n_full < (1 << 18)
    st, n, out = _static_join(lib, R, S, eps, 16)
    assert st == E.EJOIN_EOVERFLOW and n == n_full
    f = full[:n_full].cpu().numpy()
    want = _as_dict(f[:, 0], f[:, 1], f[:, 2].view(np.float32))
    o = out[:16].cpu().numpy()
    got = _as_dict(o[:, 0], o[:, 1], o[:, 2].view(np.float32))
    assert len(got) == 16 and all(k in want and want[k] == v for k, v in got.items())
    # more candidates than the fixed array holds (1.1M > 2^20 at eps = -1): EOVERFLOW with count 0
    st, n, _ = _static_join(lib, R, S, -1.0, 1 << 16)
    assert st == E.EJOIN_EOVERFLOW and n == 0
    # the array is usable again afterwards
    st, n, _ = _static_join(lib, R, S, eps, 1 << 18)
    assert st == 0 and n == n_full
