"""Learned warm start on the GPU (include/msgfem_warm.h).

* the network's forward pass, loss and gradient match the FP64 oracle
  (oracle/mlp.py), and one Adam step matches the oracle's update applied to
  the same gradient;
* on the wrinkled c1 beam (c5 workload) a network trained on eigenbases that
  the eigensolver itself produced gives start blocks closer to the converged
  spaces than the cold start, the eigensolver needs fewer iterations from
  them, and the eigenvalues it reaches match the oracle's.
"""
import numpy as np
import pytest

from parity_util import assert_eigs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

SIZES = [150, 70, 90, 130]   # several 64-wide tiles, ragged edges


def _net_problem(seed=11, B=77):
    from oracle import mlp
    rng = np.random.default_rng(seed)
    p = (rng.standard_normal(mlp.param_count(SIZES)) * 0.15).astype(np.float32)
    X = rng.standard_normal((B, SIZES[0])).astype(np.float32)
    T = rng.standard_normal((B, SIZES[-1])).astype(np.float32)
    return p, X, T


def test_net_forward_and_gradient_match_oracle():
    from oracle import mlp
    from paper_2211_13893_gb300 import Net
    p, X, T = _net_problem()
    B = X.shape[0]
    net = Net(SIZES, 128, p)
    Xd = torch.tensor(X, device="cuda")
    Td = torch.tensor(T, device="cuda")
    Y = torch.empty((B, SIZES[-1]), dtype=torch.float32, device="cuda")
    net.forward(Xd, Y, B)
    Yref, _ = mlp.forward(p.astype(np.float64), SIZES, X.astype(np.float64))
    assert np.max(np.abs(Y.cpu().numpy() - Yref)) <= 1e-5 * np.max(np.abs(Yref))
    loss, g = net.gradient(Xd, Td, B)
    loss_ref, g_ref = mlp.backward(p.astype(np.float64), SIZES, X.astype(np.float64), T.astype(np.float64))
    assert loss == pytest.approx(loss_ref, rel=1e-5)
    # per layer: weights and biases to FP32 accuracy of the largest entry
    off = 0
    for l in range(len(SIZES) - 1):
        for n in (SIZES[l + 1] * SIZES[l], SIZES[l + 1]):
            gg, gr = g[off:off + n], g_ref[off:off + n]
            assert np.max(np.abs(gg - gr)) <= 1e-4 * np.max(np.abs(gr)), (l, n)
            off += n
    assert off == g.size
    net.close()


def test_adam_step_matches_oracle_update():
    from oracle import mlp
    from paper_2211_13893_gb300 import Net
    p, X, T = _net_problem(seed=12)
    B = X.shape[0]
    net = Net(SIZES, 128, p)
    Xd = torch.tensor(X, device="cuda")
    Td = torch.tensor(T, device="cuda")
    m = np.zeros(p.size)
    v = np.zeros(p.size)
    cur = p.astype(np.float64)
    lr = 1e-3
    for t in (1, 2, 3):
        _, g = net.gradient(Xd, Td, B)           # the GPU's gradient at the current parameters
        net.adam_step(Xd, Td, B, lr)
        cur, m, v = mlp.adam_step(cur, g.astype(np.float64), m, v, t, lr)
        got = net.params().astype(np.float64)
        assert np.max(np.abs(got - cur)) <= 1e-3 * lr + 1e-6 * np.max(np.abs(cur))
        cur = got
    net.close()


def _c5_handle(tol=1e-6):
    from paper_2211_13893_gb300 import MSGFEM
    from workloads import element_angles, get_config
    cfg = get_config("c5")
    ang = torch.tensor(element_angles(cfg).reshape(-1), dtype=torch.float64, device="cuda")
    m = MSGFEM.from_config(cfg, ang, seed=5, tol=tol)
    return cfg, m


def _sample(cfg, s):
    from workloads import element_angles, wrinkle_field
    d = wrinkle_field(cfg, s)
    ang = element_angles(cfg) + d
    return (torch.tensor(ang.reshape(-1), dtype=torch.float64, device="cuda"),
            torch.tensor(d.reshape(-1), dtype=torch.float64, device="cuda"))


def test_warm_start_on_wrinkled_beam():
    from oracle import mlp
    from paper_2211_13893_gb300.warm import WarmStart
    cfg, m = _c5_handle()
    n_loc = cfg.n_loc
    ws = WarmStart(m, n_loc, hidden=(32,), seed=3)
    m.local_spaces(n_loc)
    ws.set_nominal()
    n_train, n_test = 96, 12
    X = []
    T = [[] for _ in range(m.N)]
    for s in range(n_train):
        ang, d = _sample(cfg, s)
        m.update_angles(ang)
        m.local_spaces(n_loc)
        X.append(ws.features(d))
        for j, t in enumerate(ws.targets()):
            T[j].append(t.reshape(-1))
    X = torch.stack(X)
    T = [torch.stack(t) for t in T]
    losses = ws.fit(X, T, steps=1500, lr=3e-4, batch=32)
    assert all(np.isfinite(losses))
    ang_w, ang_c, it_w, it_c = [], [], [], []
    for s in range(384, 384 + n_test):
        ang, d = _sample(cfg, s)
        m.update_angles(ang)
        ws.apply(None)
        lam_cold = m.local_spaces(n_loc).copy()
        it_c.append(sum(m.info(j)["iterations"] for j in range(m.N)))
        conv = [t.cpu().numpy() for t in ws.targets()]
        blocks = ws.predict(ws.features(d))
        ws.apply(blocks)
        lam_warm = m.local_spaces(n_loc).copy()
        it_w.append(sum(m.info(j)["iterations"] for j in range(m.N)))
        for j in range(m.N):
            assert_eigs(lam_warm[j], lam_cold[j], 1e-8, j)
        rng = np.random.default_rng(s)
        for j, (n2, nw) in enumerate(ws.sizes):
            ang_w.append(mlp.max_angle(blocks[j].cpu().numpy()[:, :nw], conv[j][:, :nw]))
            ang_c.append(mlp.max_angle(rng.standard_normal((n2, nw)), conv[j][:, :nw]))
    ws.apply(None)
    assert np.mean(ang_w) < 0.5 * np.mean(ang_c)
    assert np.mean(it_w) < np.mean(it_c)
    m.close()


def test_warm_started_eigenvalues_match_oracle():
    from oracle.coarse import run_msgfem
    from paper_2211_13893_gb300.warm import WarmStart
    cfg, m = _c5_handle()
    ws = WarmStart(m, cfg.n_loc, hidden=(32,), seed=4)
    m.local_spaces(cfg.n_loc)
    ws.set_nominal()
    ws.build()                       # untrained network: nominal blocks plus a small perturbation
    ang, d = _sample(cfg, 400)
    m.update_angles(ang)
    ws.apply(ws.predict(ws.features(d)))
    lam = m.local_spaces(cfg.n_loc)
    ws.apply(None)
    ref = run_msgfem(cfg, angles=ang.cpu().numpy().reshape(cfg.NX, cfg.NY, cfg.NZ), solver="dense")
    for j in range(m.N):
        assert_eigs(lam[j], np.asarray(ref.lam[j])[:cfg.n_loc], 1e-8, j)
    m.close()
