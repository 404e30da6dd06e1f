"""The device-side input generator writes exactly the bytes of the C generator.

Both sides are the shared input module (no identity-by-state arithmetic): the
large GPU tests and the bench draw their inputs on the device, the oracle's
checks draw them on the host, so the two must agree byte for byte.  Cases
cover padding garbage, the structured cohort's offspring and duplicates, a
variant window with an offset, and query samples with their own ids.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _both(model, samples, pad=False):
    from paper_1410_4803_gb300 import synth
    host = synth.generate(model, samples, pad_garbage=pad)
    dev = synth.generate_device(model, samples, pad_garbage=pad).cpu().numpy()
    return host, dev


def test_plain_with_padding_garbage():
    from paper_1410_4803_gb300 import synth
    for n in (1, 3, 255, 256, 1001):
        model = synth.plain_model(777, 11, maf=(0.01, 0.5), miss=0.05, hi_miss_frac=0.01)
        host, dev = _both(model, synth.Samples.base(n), pad=True)
        assert np.array_equal(host, dev), f"n={n}"


def test_structured_relatives_and_window():
    from paper_1410_4803_gb300 import synth
    model = synth.balding_nichols_model(3000, 5, n_pop=5)
    s = synth.structured_samples(600, 5, 40, 30, 5)
    host, dev = _both(model, s)
    assert np.array_equal(host, dev)
    win = model.window(1234, 999)
    host, dev = _both(win, s.take(np.arange(17, 650, 3)))
    assert np.array_equal(host, dev)


def test_config1_and_query_samples():
    from paper_1410_4803_gb300 import synth
    w = synth.plain_config1(pad_garbage=True)
    d = synth.plain_config1(pad_garbage=True, device=0)
    assert np.array_equal(w.packed, d.packed.cpu().numpy())
    panel = synth.serving_panel(n_base_per_pop=200, m=5000, n_offspring=20, n_dup=10)
    q, qs = synth.serving_queries(panel, 77, request_id=3)
    got = synth.generate_device(panel.model, qs).cpu().numpy()
    assert np.array_equal(q, got)
