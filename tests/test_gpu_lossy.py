"""GPU lossy boson sampling (pq_bs_probs_lossy) against the oracle on the same
seeded lossy interferometer V diag(sqrt(eta)) W (Sec. 3.2.4)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2403_04006_gb300 import api, pq  # noqa: E402
from paper_2403_04006_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pq.load_library()
    return torch.device("cuda:0")


def patterns_upto(n, m):
    def comp(k, mm):
        if mm == 1:
            return [[k]]
        return [[v] + r for v in range(k + 1) for r in comp(k - v, mm - 1)]
    out = []
    for k in range(n + 1):
        out += comp(k, m)
    return np.array(out, dtype=np.int32)


@pytest.mark.parametrize("m,s", [(5, [1, 1, 0, 1, 0]), (6, [2, 0, 1, 0, 1, 0])])
def test_lossy_probabilities_match_oracle(dev, m, s):
    rng = np.random.default_rng(77 + m)
    V, Wm = W.haar_unitary(m, rng), W.haar_unitary(m, rng)
    eta = rng.uniform(0.2, 0.95, m)
    s = np.array(s, dtype=np.int32)
    t = patterns_upto(int(s.sum()), m)
    got = api.bs_probs_lossy(torch.from_numpy(V).to(dev), torch.from_numpy(eta).to(dev),
                             torch.from_numpy(Wm).to(dev), s, t).cpu().numpy()
    ref = O.lossy_probs(V, eta, Wm, s, t)
    assert abs(got.sum() - 1.0) <= 1e-13
    big = ref > 1e-12
    assert np.abs(got[big] - ref[big]).max() <= 1e-10 * np.abs(ref[big]).max()
    assert (np.abs(got - ref) <= 1e-10 * ref + 1e-16).all()


def test_lossy_rejects_too_many_photons(dev):
    m = 3
    I = torch.eye(m, dtype=torch.complex128, device=dev)
    eta = torch.ones(m, dtype=torch.float64, device=dev)
    with pytest.raises(pq.PQError) as e:
        api.bs_probs_lossy(I, eta, I, [1, 0, 0], [[1, 1, 0]])
    assert e.value.code == pq.PQ_ERR_ARG


def test_lossy_plan_runs_match_the_one_shot_call(dev):
    """A lossy plan made once evaluates, run after run, what the one-shot call
    gives for each new interferometer (same schedule, same bits), and the
    oracle's probabilities."""
    m = 5
    s = np.array([1, 1, 0, 1, 0], dtype=np.int32)
    t = patterns_upto(3, m)
    plan = api.LossyPlan(m, s, t)
    rng = np.random.default_rng(91)
    for _ in range(3):
        V, Wm = W.haar_unitary(m, rng), W.haar_unitary(m, rng)
        eta = rng.uniform(0.2, 0.95, m)
        Vd, Wd, ed = (torch.from_numpy(x).to(dev) for x in (V, Wm, eta))
        got = plan.run(Vd, ed, Wd).cpu().numpy()
        want = api.bs_probs_lossy(Vd, ed, Wd, s, t).cpu().numpy()
        assert np.array_equal(got, want)
        ref = O.lossy_probs(V, eta, Wm, s, t)
        assert (np.abs(got - ref) <= 1e-10 * ref + 1e-16).all()
    plan.close()
    empty = api.LossyPlan(m, s, np.zeros((0, m), dtype=np.int32))
    I = torch.eye(m, dtype=torch.complex128, device=dev)
    assert empty.run(I, torch.ones(m, dtype=torch.float64, device=dev), I).numel() == 0
    with pytest.raises(pq.PQError) as e:
        api.LossyPlan(m, s, [[1, 1, 1, 1, 0]])  # more photons than the input
    assert e.value.code == pq.PQ_ERR_ARG
