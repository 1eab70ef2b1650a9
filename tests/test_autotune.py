"""The autotuner's candidate spaces (host logic) and, on the GPU, that it
leaves the handle on the fastest measured tuning without changing results."""
import json

import numpy as np
import pytest

from paper_1412_4825_gb300 import autotune as AT


def test_candidates_enumerate_the_product():
    c = AT.candidates({"b": [1, 2], "a": [3, 4, 5]})
    assert len(c) == 6
    assert {json.dumps(x, sort_keys=True) for x in c} == {
        json.dumps({"a": a, "b": b}, sort_keys=True) for a in (3, 4, 5) for b in (1, 2)}
    for kind, space in AT.SPACES.items():
        cands = AT.candidates(space)
        assert len(cands) == int(np.prod([len(v) for v in space.values()])), kind
        assert all(set(x) == set(space) for x in cands)


@pytest.mark.gpu
def test_autotune_picks_fastest_and_keeps_results():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_4825_gb300 import brng as B

    dev = torch.device("cuda:0")
    stream = torch.cuda.Stream()

    def run(tuned):
        h = B.Handle(7, 1)
        st = B.triangle_state(300, device=dev)
        mom = torch.zeros((300, 5), dtype=torch.float64, device=dev)
        launch = lambda: B.brng_gibbs_run(h.h, B.MODEL_TRIANGLE, 0, 300, 50, None, st, mom, stream)  # noqa: E731
        if tuned:
            tune, ms, table = AT.autotune(h, launch, AT.SPACES["triangle"], stream, "test-triangle-300x50")
            assert ms == min(table.values())
            assert h.tuning["lanes_per_chain"] == tune["lanes_per_chain"]
            assert h.tuning["buf_len"] == tune["buf_len"]
            st.copy_(B.triangle_state(300, device=dev))
            mom.zero_()
        launch()
        torch.cuda.synchronize()
        out = (st.clone(), mom.clone())
        h.close()
        return out

    a, b = run(False), run(True)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
