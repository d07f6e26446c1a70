"""Continuous-batching server: admission policy (CPU) and results that do not
depend on the mix a request is served in (GPU)."""
import collections

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2607_10280_b300 import synth  # noqa: E402


def test_admission_policy_respects_count_and_bytes():
    from paper_2607_10280_b300.serving import form_wave, image_footprint
    reqs = collections.deque([{"b": b} for b in (5, 3, 4, 10, 1, 1)])
    wave, foot = form_wave(reqs, max_images=10, room=12, footprint=lambda r: r["b"])
    assert [r["b"] for r in wave] == [5, 3, 4] and foot == 12 and len(reqs) == 3
    wave, foot = form_wave(reqs, max_images=1, room=100, footprint=lambda r: r["b"])
    assert [r["b"] for r in wave] == [10] and len(reqs) == 2
    wave, foot = form_wave(reqs, max_images=8, room=0, footprint=lambda r: r["b"])
    assert wave == [] and foot == 0 and len(reqs) == 2        # nothing fits: nothing admitted
    # footprint: sites (2 ld^2) + environments (ld^2) complex values per qubit
    assert image_footprint(7, 16) == 49 * 3 * 16 * 16 * 8
    assert image_footprint(2, 64) == 4 * 3 * 4 * 4 * 8         # bond limited by 2^(n/2) = 4
    assert image_footprint(7, 16, "fp64") == 2 * image_footprint(7, 16)
    # with the depth: left environments of an operator-product image (L = 4, chi = 16),
    # the complex128 chain of a truncating one (L = 4, chi = 8), neither at L = 3, chi = 8
    assert image_footprint(7, 16, "mixed", 4) == 49 * 4 * 16 * 16 * 8
    assert image_footprint(7, 8, "mixed", 4) == 49 * 3 * 8 * 8 * 8 + 49 * 2 * 8 * 8 * 16
    assert image_footprint(7, 8, "mixed", 3) == 49 * 4 * 8 * 8 * 8
    assert image_footprint(7, 8, "fp64", 4) == 49 * 3 * 8 * 8 * 16


@pytest.mark.gpu
def test_results_do_not_depend_on_the_mix():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle import pipeline as o_pipe
    from paper_2607_10280_b300 import build
    from paper_2607_10280_b300.serving import Request, Server, image_footprint
    build.build()
    params_np = synth.circuit_params(3, 64, seed=17)
    params = torch.tensor(params_np, dtype=torch.float64, device="cuda")
    m7 = 84
    abd = torch.tensor(synth.observable_params(m7), dtype=torch.float32, device="cuda")
    W, b = synth.linear_params(784, m7)
    epi = {7: (abd, torch.tensor(W, dtype=torch.float32, device="cuda"),
               torch.tensor(b, dtype=torch.float32, device="cuda"))}
    rng = np.random.default_rng(3)
    spec = [(int(rng.integers(4, 9)), int(rng.integers(1, 4)), int(rng.choice([4, 8]))) for _ in range(40)]
    spec += [(7, 2, 8)] * 6
    pix = [synth.garment_pixels(1, p, seed=500 + i)[0] for i, (p, _, _) in enumerate(spec)]
    budget = 6 * image_footprint(8, 8) + 1
    srv = Server(params, epi, slots=3, max_images_per_wave=8, budget_bytes=budget, max_p=8, max_chi=8)
    srv.start()
    reqs = [srv.submit(Request(p, L, chi, pix[i])) for i, (p, L, chi) in enumerate(spec)]
    for r in reqs:
        assert r.event.wait(120)
    srv.stop()
    assert srv.waves > 1 and srv.max_inflight_bytes <= budget
    # requests that run a truncating (complex128) chain were served by the long lane only
    from paper_2607_10280_b300.flops import lossy
    assert any(lossy(r.p, r.L, r.chi) for r in reqs) and any(not lossy(r.p, r.L, r.chi) for r in reqs)
    for r in reqs:
        assert r.lane == ("long" if lossy(r.p, r.L, r.chi) else "short"), (r.p, r.L, r.chi, r.lane)
    assert all(w[3] > 0 and w[4] >= 0 for w in srv.wave_log)
    # every request again, alone in its own wave
    alone = Server(params, epi, slots=1, max_images_per_wave=1, max_p=8, max_chi=8)
    alone.start()
    solo = [alone.submit(Request(p, L, chi, pix[i])) for i, (p, L, chi) in enumerate(spec)]
    for r in solo:
        assert r.event.wait(120)
    alone.stop()
    for r, s in zip(reqs, solo):
        assert np.array_equal(r.pauli, s.pauli)                  # bit-identical alone and in the mix
        if r.p == 7:
            assert np.array_equal(r.features, s.features) and np.array_equal(r.output, s.output)
    checked = 0
    for i in (0, 5, 9, 40):
        p, L, chi = spec[i]
        ref, st = o_pipe.pauli_cache(pix[i], p, L, chi, "ladder", params_np, return_state=True)
        if st.min_gap < 1e-6:
            continue                      # near-tie at a truncation cut: no unique answer
        assert np.max(np.abs(reqs[i].pauli - ref)) < 1e-5
        checked += 1
    assert checked >= 2
