"""The learned selector's device code against its CPU oracle, and what the
trained network gains over the fixed default on held-out matrices."""
import numpy as np
import pytest

import synth
from oracle import selector as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1504_06474_gb300 import _build
    _build.build()
    return torch.device("cuda:0")


def _mats():
    yield synth.workload("uniform4096")[0]
    yield synth.banded(3000, 9, seed=1)
    yield synth.blockdiag(5000, 32, 100, seed=2)
    yield synth.long_rows(20000, 3, 5000, seed=3)
    yield synth.rmat_clipped(30000, 8, seed=4)
    yield synth.CSR(50, 50, np.zeros(51, np.int32), np.zeros(0, np.int32), np.zeros(0))


def test_features_match_oracle(dev):
    from paper_1504_06474_gb300 import selector as S
    for A in _mats():
        rp = torch.as_tensor(A.row_ptr, device=dev)
        f = S.device_features(rp, A.m, A.n, A.nnz).cpu().numpy().astype(np.float64)
        ref = O.features(A.row_ptr, A.n)
        assert np.allclose(f, ref, rtol=1e-6, atol=1e-7), (A.name, f, ref)


def test_mlp_kernels_match_oracle(dev):
    from paper_1504_06474_gb300 import ssspmv as C
    rng = np.random.default_rng(7)
    F, H1, H2, K, B = 16, 64, 64, 10, 37
    p = rng.normal(0, 0.3, O.sizes(F, H1, H2, K)).astype(np.float32)
    X = rng.normal(0, 1, (B, F)).astype(np.float32)
    T = rng.normal(3, 1, (B, K)).astype(np.float32)
    T[3, 4] = np.nan
    pd, Xd, Td = (torch.as_tensor(a, device=dev) for a in (p, X, T))
    scratch = torch.empty(C.ssspmv_mlp_scratch_floats(B, F, H1, H2, K), dtype=torch.float32,
                          device=dev)
    out = torch.empty((B, K), dtype=torch.float32, device=dev)
    C.check(C.ssspmv_mlp_forward(pd, Xd, B, F, H1, H2, K, scratch, out), "forward")
    ref_out, _ = O.forward(p.astype(np.float64), X.astype(np.float64), F, H1, H2, K)
    assert np.allclose(out.cpu().numpy(), ref_out, rtol=1e-4, atol=1e-4)
    g = torch.empty_like(pd)
    loss = torch.empty(1, dtype=torch.float32, device=dev)
    C.check(C.ssspmv_mlp_backward(pd, Xd, Td, B, F, H1, H2, K, scratch, g, loss), "backward")
    ref_loss, ref_g = O.loss_and_grad(p.astype(np.float64), X.astype(np.float64),
                                      T.astype(np.float64), F, H1, H2, K)
    assert np.isclose(float(loss.item()), ref_loss, rtol=1e-4)
    gh = g.cpu().numpy()
    assert np.max(np.abs(gh - ref_g)) <= 1e-4 * max(1.0, np.max(np.abs(ref_g)))
    m1 = torch.zeros_like(pd)
    m2 = torch.zeros_like(pd)
    C.check(C.ssspmv_mlp_adam(pd, g, m1, m2, pd.numel(), 1e-2, 0.9, 0.999, 1e-8, 1e-3, 1), "adam")
    ref_p, _, _ = O.adam_step(p.astype(np.float64), gh.astype(np.float64), np.zeros(p.size),
                              np.zeros(p.size), 1e-2, wd=1e-3, t=1)
    assert np.allclose(pd.cpu().numpy(), ref_p, rtol=1e-5, atol=1e-6)
    cls = torch.empty(B, dtype=torch.int32, device=dev)
    C.check(C.ssspmv_mlp_select(pd, Xd, B, F, H1, H2, K, scratch, cls), "select")
    ref_out2, _ = O.forward(ref_p, X.astype(np.float64), F, H1, H2, K)
    # the argmin of the (updated) predictions, away from near ties
    srt = np.sort(ref_out2, axis=1)
    clear = srt[:, 1] - srt[:, 0] > 1e-3
    assert np.array_equal(cls.cpu().numpy()[clear], ref_out2.argmin(axis=1)[clear])


def test_trained_selector_beats_the_fixed_default(dev):
    """Measured on held-out matrices: the network's choices against always
    running the default class, and against the best class per matrix."""
    from paper_1504_06474_gb300 import selector as S
    tr = S.dataset_specs(150, seed=101, m_lo=10_000, m_hi=400_000)
    te = S.dataset_specs(50, seed=505, m_lo=10_000, m_hi=400_000)
    Xtr, Ttr = S.collect(tr, dev, reps=3)
    Xte, Tte = S.collect(te, dev, reps=3)
    params = S.train(Xtr, S.targets(Ttr), dev, steps=3000)
    rep = S.evaluate(S.select(params, Xte, dev), Tte)
    print("held-out: selector regret %.3f (default %.3f), geomean speedup over default %.3f "
          "(best possible %.3f)" % (rep["mean_regret"], rep["default_mean_regret"],
                                    rep["geomean_speedup_vs_default"],
                                    rep["geomean_speedup_oracle_choice_vs_default"]))
    assert rep["mean_regret"] < rep["default_mean_regret"]
    assert rep["geomean_speedup_vs_default"] > 1.0


def test_adam_kernel_over_several_steps_with_decay(dev):
    """ssspmv_mlp_adam against the oracle's Adam for steps t = 1..6 with L2
    decay, carrying the moments from step to step (the bias corrections at
    t > 1 and the decay term are exercised, not only the first step)."""
    from paper_1504_06474_gb300 import ssspmv as C
    rng = np.random.default_rng(21)
    n = 1000
    p = rng.normal(0, 1, n).astype(np.float32)
    grads = rng.normal(0, 0.5, (6, n)).astype(np.float32)
    pd = torch.as_tensor(p, device=dev)
    m1d = torch.zeros(n, dtype=torch.float32, device=dev)
    m2d = torch.zeros(n, dtype=torch.float32, device=dev)
    ref_p = p.astype(np.float64)
    ref_m1 = np.zeros(n)
    ref_m2 = np.zeros(n)
    lr, wd = 3e-2, 5e-2
    # the kernel receives the hyperparameters as FP32 numbers (1 - float(0.999)
    # is 1.3e-5 away from 0.001): the oracle takes the same rounded values
    f32 = lambda v: float(np.float32(v))
    hp = dict(b1=f32(0.9), b2=f32(0.999), eps=f32(1e-8), wd=f32(wd))
    for t in range(1, 7):
        gd = torch.as_tensor(grads[t - 1], device=dev)
        C.check(C.ssspmv_mlp_adam(pd, gd, m1d, m2d, n, lr, 0.9, 0.999, 1e-8, wd, t), "adam")
        ref_p, ref_m1, ref_m2 = O.adam_step(ref_p, grads[t - 1].astype(np.float64), ref_m1,
                                            ref_m2, f32(lr), t=t, **hp)
        # FP32 kernel against the FP64 oracle: a few FP32 roundings per step
        assert np.allclose(m1d.cpu().numpy(), ref_m1, rtol=1e-5, atol=1e-7), t
        assert np.allclose(m2d.cpu().numpy(), ref_m2, rtol=1e-5, atol=1e-9), t
        assert np.allclose(pd.cpu().numpy(), ref_p, rtol=1e-5, atol=1e-6), t
    # the decay changed the result (the same steps without it land elsewhere)
    q = p.astype(np.float64)
    a = np.zeros(n)
    b = np.zeros(n)
    for t in range(1, 7):
        q, a, b = O.adam_step(q, grads[t - 1].astype(np.float64), a, b, lr, wd=0.0, t=t)
    assert np.max(np.abs(q - ref_p)) > 1e-4
