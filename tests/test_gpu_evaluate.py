"""The Sec. 4.1 search through the CUDA detector on labelled synthetic
windows (Sec. 4.2's F1 at IoU 0.5): thresholds found inside Table 2's ranges
detect the generated drones on held-out windows, where Table 2's own values
(chosen on the paper's recordings) flag the noise as well; and
ddhf_set_params gives the same boxes as a context created with those
parameters."""
import numpy as np
import pytest
import torch

from paper_2603_08386_gb300 import ddhf, evaluate, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2603_08386_gb300 import build
    build.build()
    ddhf.load()
    assert torch.cuda.is_available()
    yield


def test_set_params_equals_fresh_context():
    s = synth.labelled_scene(7)
    prm = ddhf.default_params(tau_sf=0.42, tau_comb=4.0, M=8, d=1, h_min=3, n_min=4,
                              A_min=20, alpha=4.0)
    ev = ddhf.events_to_device(s)
    a = ddhf.Context(s.W, s.H, s.grid, None, max_events=s.n)
    a.detect(*ev, s.t0, s.window_us)
    a.set_params(prm)
    bx_a, nb_a, m_a = a.detect(*ev, s.t0, s.window_us, want_mask=True)
    b = ddhf.Context(s.W, s.H, s.grid, prm, max_events=s.n)
    bx_b, nb_b, m_b = b.detect(*ev, s.t0, s.window_us, want_mask=True)
    assert int(nb_a.item()) == int(nb_b.item()) >= 1
    n = int(nb_a.item())
    np.testing.assert_array_equal(bx_a[:n].cpu().numpy(), bx_b[:n].cpu().numpy())
    assert torch.equal(m_a, m_b)
    with pytest.raises(ddhf.DDHFError):
        a.set_params(ddhf.default_params(M=0))
    a.stats()
    b.stats()
    a.close()
    b.close()


def test_search_beats_table2_on_held_out_windows():
    val = evaluate.Evaluator([synth.labelled_scene(300 + i) for i in range(3)])
    test = evaluate.Evaluator([synth.labelled_scene(400 + i) for i in range(4)])
    t2 = ddhf.default_params()
    f_t2 = test.f1(t2)
    # 30 uniformly random points, then 90 expected-improvement steps (one
    # detection of each validation window per evaluation); the F1 surface is
    # flat almost everywhere, so the budget has to reach the narrow region
    # where drones and noise separate
    best, f_val, hist = evaluate.tune(val, n_init=30, n_iter=90, seed=0)
    assert len(hist) == 120
    f_test = test.f1(evaluate.params_of(best))
    print(f"Table 2 F1 {f_t2:.3f}; tuned {best} val F1 {f_val:.3f} test F1 {f_test:.3f}")
    assert f_val >= 0.8
    assert f_test >= 0.7 and f_test > f_t2 + 0.3
    val.close()
    test.close()
