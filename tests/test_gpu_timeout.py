"""Failure detection on the GPU: a device-side wait that runs out.

Every wait of the tensor-core kernels is bounded by the context's
timeout_cycles.  With a bound of one cycle the waits of a large contraction
(d = 4096: each 128 x 256 tile needs tens of microseconds of MMAs before the
epilogue can read it) run out; the call must return EJOIN_ETIMEOUT, and the
kernel must have let its issued copies and MMAs complete and freed its tensor
memory, so that the same context, given the default bound again, computes a
join that matches the FP64 oracle.  No fault and no hang is involved: the
kernels return normally with an error word the host reads.
"""
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


def gauss(seed, n, d):
    return np.random.default_rng(seed).standard_normal((n, d)).astype(np.float32)


@pytest.mark.parametrize("prec", ["bf16", "fp8", "tf32"])
def test_wait_runs_out_then_context_recovers(prec):
    big_R = torch.from_numpy(gauss(1, 6000, 4096)).cuda()
    big_S = torch.from_numpy(gauss(2, 5000, 4096)).cuda()
    R, S = gauss(3, 700, 200), gauss(4, 900, 200)
    eps = 0.15
    with pkg.Ctx(device=0, prec=prec) as ctx:
        pkg.ejoin_set_timeout(ctx, 1)
        with pytest.raises(pkg.EJoinError) as ei:
            pkg.ejoin_threshold(ctx, big_R, big_S, 0.5)
        assert ei.value.status == E.EJOIN_ETIMEOUT
        # the E-selection scan bounds its waits the same way
        with pytest.raises(pkg.EJoinError) as ei:
            pkg.ejoin_eselect(ctx, big_R, big_S[:64].contiguous(), 0.5)
        assert ei.value.status == E.EJOIN_ETIMEOUT
        torch.cuda.synchronize()  # the CUDA context is intact
        pkg.ejoin_set_timeout(ctx, 0)
        res = pkg.ejoin_threshold(ctx, torch.from_numpy(R).cuda(), torch.from_numpy(S).cuda(), eps)
        gi = res.i.cpu().numpy().view(np.uint32)
        gj = res.j.cpu().numpy().view(np.uint32)
        gs = res.sim.cpu().numpy()
    oi, oj, os_ = oracle.join(R, S, eps)
    assert len(oi) > 1000
    compare(R, S, eps, gi, gj, gs, oi, oj, os_)


def test_set_timeout_rejects_null_context():
    lib = E.load_library()
    assert lib.ejoin_set_timeout(None, 5) == E.EJOIN_EINVAL
