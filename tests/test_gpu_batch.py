"""Uneven instances in one graph and the schedule autotuner, on the GPU.

The 8 PDE-like lattice instances (m in {14, 16, 18}, s up to 2048, tau up to 4096, 4 shifts
each) go to the library in one call, which runs them on parallel internal streams; the
Integrator captures that call as one CUDA graph.  Every instance's estimates are compared with
the oracle's stored full-size values.  The autotuner times the fine band's schedules and caches
the fastest; results under the tuned schedule are compared with the oracle."""
import numpy as np
import pytest
import torch

from oracle import qmc_oracle as O
from paper_2305_11645_gb300 import _lib as L
from paper_2305_11645_gb300 import api
from paper_2305_11645_gb300 import inputs as I
from tests.gpu_common import golden, integrand, need_gpu, norm_rel

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    need_gpu()
    api.tune_clear()
    yield
    api.tune_clear()


@pytest.mark.parametrize("precision", ["split", None])
def test_uneven_instances_in_one_graph(precision):
    ps = [I.c4(i) for i in range(len(I.C4_INSTANCES))]
    rules = [api.Rule.from_problem(p) for p in ps]
    As = [torch.from_numpy(p.A).to(DEV) for p in ps]
    fs = [integrand(p) for p in ps]
    it = api.Integrator(rules, As, fs, backward=False, graph=True, precision=precision)
    est1 = it.run()[0].clone()
    est2 = it.run()[0].clone()
    torch.cuda.synchronize()
    assert torch.equal(est1, est2)
    est = est1.cpu().numpy()
    tol = 1e-6 if precision == "split" else 2e-5
    off = 0
    for i, p in enumerate(ps):
        g = golden("c4")[i]
        got = est[off:off + p.R_eff + 1]
        Q = np.array(g["Q"])
        assert np.all(np.abs(got[:-1] - Q) <= tol * np.abs(Q)), (i, got, Q)
        assert abs(got[-1] - g["mean"]) <= tol * abs(g["mean"])
        off += p.R_eff + 1
    # the eager call on the caller's stream gives the same numbers
    eager = api.integrate(rules, As, fs, precision=precision).cpu().numpy()
    assert np.array_equal(eager, est)


def test_batched_backward_matches_single_calls():
    ps = [I.random_problem(40 + i, kind=I.LATTICE if i % 2 else I.DIGITAL_NET, m=9 + i, s=40 + 13 * i,
                           tau=33 + 20 * i, R=1 + i % 3, dtype=np.float32, f_kind=I.F_LOGSUMEXP) for i in range(4)]
    rules = [api.Rule.from_problem(p) for p in ps]
    As = [torch.from_numpy(p.A).to(DEV) for p in ps]
    fs = [integrand(p) for p in ps]
    up = torch.tensor([1.0, 0.5, 2.0, -1.0], dtype=torch.float64, device=DEV)
    grads = api.integrate_backward(rules, As, fs, up, precision="split")
    for i, (rule, A, f, p) in enumerate(zip(rules, As, fs, ps)):
        single = api.integrate_backward(rule, A, f, up[i:i + 1], precision="split")[0]
        assert torch.equal(grads[i], single)
        assert norm_rel(grads[i].double().cpu().numpy(), float(up[i]) * O.grad(p)) <= 2e-5


@pytest.mark.parametrize("precision", ["split", "fp32"])
def test_autotune_then_parity(precision, tmp_path):
    p = I.c2(m=13, s=256, dtype=np.float32)
    rule = api.Rule.from_problem(p)
    A = torch.from_numpy(p.A).to(DEV)
    f = integrand(p)
    n = api.autotune(rule, A, f, precision=precision)
    assert n >= 2
    est = api.integrate(rule, A, f, precision=precision).cpu().numpy()
    Q, mean = O.estimate(p)
    assert abs(est[-1] - mean) <= 2e-5 * abs(mean)
    G = api.integrate_backward(rule, A, f, torch.ones(1, dtype=torch.float64, device=DEV), precision=precision)[0]
    assert norm_rel(G.cpu().numpy(), O.grad(p)) <= 2e-5
    path = tmp_path / "sched.txt"
    api.tune_save(str(path))
    api.tune_clear()
    assert api.tune_load(str(path)) >= 1
    est2 = api.integrate(rule, A, f, precision=precision).cpu().numpy()
    assert np.array_equal(est, est2)                         # the reloaded schedule is the same plan
    L.device_status(clear=True)
