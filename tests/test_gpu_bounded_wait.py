"""Failure detection without a GPU fault: a device-side wait that never completes gives up
after its poll limit, the library reports SLAR_ETIMEOUT, and the CUDA context stays usable
(the tensor-core evaluator's mbarrier waits use the same bounded loop)."""
import numpy as np
import pytest

from oracle import sl
from paper_2606_29027_b300 import inputs, slar

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import test_gpu_parity as P  # noqa: E402


def test_wait_that_never_completes_gives_up_and_the_context_stays_usable():
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    assert slar.wait_probe(1024, status) == slar.SLAR_ETIMEOUT
    assert int(status.item()) == 1
    # bad limits are rejected before any launch
    assert slar.wait_probe(0, status) == slar.SLAR_EINVAL
    # the context keeps working: an entry evaluation against the oracle
    N, ranks = (16, 16, 16, 16), (5, 6, 4, 7, 8, 9)
    h, _, _ = P.rand_state(N, ranks, 41)
    ctx, g = P.ctx_for(N)
    P.load(ctx, h)
    E = inputs.random_field(N[:2], 2, 0.4, seed=42)
    idx = inputs.random_tuples(N, 777, seed=43)
    out = torch.zeros(idx.shape[0], dtype=torch.float64, device="cuda")
    ctx.sl_eval(0.5, P.dev(E), P.dev(idx, torch.int32), out)
    want = sl.sl_eval(h, E, 0.5, idx, g)
    assert P.relerr(out.cpu().numpy(), want) < 1e-12
    ctx.close()
