"""Failure path of the tensor-core stage, made to happen on purpose without a
fault: a tiny spin limit makes the Gram kernel's bounded mbarrier waits run
out.  The kernel must report the timeout through the status word (the
correlation integral then returns n_rechecked = -2), drain its own copies and
tensor-core work, and leave the context usable: the next call with the
default limit is exact again."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def p():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2203_14742_b300 as pk
    return pk


def test_spin_limit_timeout_is_reported_and_context_recovers(p):
    X1 = W.clustered_patterns(256, 8192, 41)
    X2 = W.clustered_patterns(200, 8192, 42)
    t1, t2 = torch.from_numpy(X1).cuda(), torch.from_numpy(X2).cuda()
    ref = p.cil(t1, t2, b=1.2, M=16)
    torch.cuda.synchronize()
    assert int(ref["n_rechecked"]) >= 0
    try:
        p.lib().rd_set_spin_limit(1)
        for _ in range(2):
            bad = p.cil(t1, t2, b=1.2, M=16)
            torch.cuda.synchronize()
            assert int(bad["n_rechecked"]) == -2
    finally:
        p.lib().rd_set_spin_limit(0)
    for _ in range(2):
        again = p.cil(t1, t2, b=1.2, M=16)
        torch.cuda.synchronize()
        assert int(again["n_rechecked"]) >= 0
        assert torch.equal(again["bins"], ref["bins"])
        assert torch.equal(again["counts"], ref["counts"])
    o = oracle.cil(X1, X2, b=1.2, M=16)
    assert np.array_equal(again["counts"].cpu().numpy(), o["counts"])
