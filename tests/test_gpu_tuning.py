"""Every launch variant the autotuner can pick gives the same sums (GPU):
counts bit-exact, FP64 sums equal up to the rounding of their grouping."""
import numpy as np
import pytest

import paper_1612_07717_gb300 as G
from paper_1612_07717_gb300 import autotune as T
from paper_1612_07717_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("integ", [G.SE, G.GL, G.BAOAB])
def test_all_variants_agree(integ):
    d = W.bl600(integ)
    p = G.make_params(d)
    lm = d["level_min"]
    reqs = [(lm + 3, 0, 20001), (lm + 1, 5, 80000), (lm, 0, 300000)]
    ref = [G.level_sums(l, n, integ, p, 9, path_offset=f) for l, f, n in reqs]
    saved = T.get_tuning(integ, G.FP32)
    try:
        for var in (1, 3, 4, 12, 13):
            for ipb in (4, 64):
                T.set_tuning(integ, G.FP32, var, ipb, 0)
                got = G.multilevel_sums(reqs, integ, p, 9)
                for a, b in zip(got, ref):
                    assert a["n"] == b["n"]
                    assert np.array_equal(np.array(a["sum"][1]), np.array(b["sum"][1]))
                    assert np.allclose(a["sum"][0], b["sum"][0], rtol=1e-11)
        T.set_tuning(integ, G.FP32, 4, 16, 2)               # capped resident blocks
        got = G.multilevel_sums(reqs, integ, p, 9)
        assert [a["n"] for a in got] == [b["n"] for b in ref]
    finally:
        T.set_tuning(integ, G.FP32, saved["variant"], saved["items_per_block"],
                     saved["blocks_per_sm"])


def test_tuning_rejects_bad_values():
    L = G.lib()
    assert L.mlmc_set_tuning(G.GL, G.FP32, 2, 16, 0) == G.EINVAL
    assert L.mlmc_set_tuning(G.GL, G.FP64, 4, 16, 0) == G.EINVAL
    assert L.mlmc_set_tuning(G.GL, G.FP32, 3, 0, 0) == G.EINVAL
