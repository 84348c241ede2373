"""The allocation-free elimination selection (lg_elim_select_noalloc).

It exists for callers that must not allocate device memory during a call
(memory pools that must not grow, callbacks or runtimes that forbid
cudaMalloc, loops that cannot take an allocation's stall). Its scratch lives
in a fixed device array shared by all calls, so this file is collected last
and checks two calls in a row: the second must not see the first one's
leftovers. Results must equal lg_elim_select and the oracle's selection
(Section 3.4, Algorithm 2) bit for bit (integer work).
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SEED = 0x5EED


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_noalloc_matches_allocating_selection_twice(torch_cuda, lgmod, oracle, inputs):
    torch = torch_cuda
    graphs = [inputs.chung_lu(200000, m_target=1000000, seed=5), inputs.grid2d(300, 300)]
    for g in graphs:  # two calls in a row on different graphs share the scratch
        rp, cl = dev(torch, g.rowptr), dev(torch, g.col)
        ref = torch.zeros(g.n, dtype=torch.uint8, device="cuda")
        nf_ref = lgmod.lg_elim_select(g.n, rp, cl, 4, SEED, ref)
        out = torch.full((g.n,), 7, dtype=torch.uint8, device="cuda")
        nf = lgmod.lg_elim_select_noalloc(g.n, rp, cl, 4, SEED, out)
        assert nf == nf_ref
        assert torch.equal(out, ref)
        nf2 = lgmod.lg_elim_select_noalloc(g.n, rp, cl, 4, SEED, out)
        assert nf2 == nf_ref and torch.equal(out, ref)
        want = oracle.elim_select(g, 4, SEED).astype(np.uint8)
        np.testing.assert_array_equal(out.cpu().numpy(), want)
        assert nf == int(want.sum())


def test_noalloc_rejects_too_large(torch_cuda, lgmod, inputs):
    torch = torch_cuda
    n = (1 << 20) + 1
    rp = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    cl = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.zeros(n, dtype=torch.uint8, device="cuda")
    with pytest.raises(lgmod.LGError) as e:
        lgmod.lg_elim_select_noalloc(n, rp, cl, 4, SEED, out)
    assert e.value.status == lgmod.ERR_INVALID and "1048576" in str(e.value)
