"""Host-side failure paths that leave the GPU and the context usable.

Allocation failure is made on the host: a context memory limit below what
the graph needs makes the call return EF_ERR_OOM before it frees or
allocates anything; raising the limit lets the same context finish the same
graph.  Malformed graphs (EF_ERR_GRAPH) are covered by the parity tests.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def test_memory_limit_gives_oom_and_leaves_the_context_usable():
    import torch
    import paper_2306_00606_gb300 as ef
    g = synth.barabasi_albert(20000, 5, 11)
    rp = torch.from_numpy(g.row_ptr).cuda()
    ci = torch.from_numpy(g.col_idx).cuda()
    ref = oracle.alg1(g)
    with ef.Context(0) as ctx:
        ctx.set_memory_limit(1 << 20)
        with pytest.raises(ef.EfError) as ei:
            ctx.compute(rp, ci, precision="fp64")
        assert ei.value.code == ef.EF_ERR_OOM and "memory limit" in str(ei.value)
        # a graph that fits under the cap still runs on the same context
        small = synth.erdos_renyi(200, 0.02, 3)
        out = ctx.compute(torch.from_numpy(small.row_ptr).cuda(), torch.from_numpy(small.col_idx).cuda(),
                          precision="fp64")
        np.testing.assert_allclose(out["ef"].cpu().numpy(), oracle.alg1(small)["EF"], rtol=1e-9, atol=1e-12)
        ctx.set_memory_limit(0)
        out = ctx.compute(rp, ci, precision="fp64", outputs=("ef", "s"))
        np.testing.assert_array_equal(out["s"].cpu().numpy(), ref["S"])
        np.testing.assert_allclose(out["ef"].cpu().numpy(), ref["EF"], rtol=1e-9, atol=1e-12)
        # a cap above what is held changes nothing
        ctx.set_memory_limit(1 << 40)
        out = ctx.compute(rp, ci, precision="fp32c")
        np.testing.assert_allclose(out["ef"].cpu().numpy(), ref["EF"], rtol=0, atol=2e-5)
