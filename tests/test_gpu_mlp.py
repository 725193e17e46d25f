"""The learned part: the MLP surrogate inverse CDF trained with the
library's FP16 tensor-core kernels and evaluated in binary16 inference
arithmetic, checked against the oracle.

* gradients of one full pass against the oracle's manual backprop;
* the inference (approx_icdf with the MLP, and the tabulated network the
  level kernels read) bit for bit against the oracle's binary16 reading, and
  within its error of the FP64 network;
* one Adam step against the oracle's Adam on the same minibatch (the
  minibatch indices come from the same counter-based generator);
* training on 2^20 oracle pairs beats the piecewise-linear table in
  E|Z - Z~|^2 (the quantity of Lemma 3.1);
* inside the four-way difference: per-path agreement with the FP64 oracle
  within the workload's 2e-3 at l = 2, 6, 10, 12 and bit for bit with the
  oracle's binary16 emulation (network and Euler), lower four-way variance
  than the table (what the network gains), and unbiased nested level means.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
from oracle import mlp as OM  # noqa: E402
import paper_2012_09739_gb300 as M  # noqa: E402
from workloads import mlp_initial_weights, uniform_grid_sample  # noqa: E402

SEED = 1234


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _pairs(n, seed):
    u = uniform_grid_sample(n, seed)
    v = np.minimum(u, 1.0 - u)
    return u, -O.ndtri(v)        # targets |Phi^-1(v)| from the oracle


def _perturbed_weights(seed=7):
    w = mlp_initial_weights(1234)
    rng = np.random.default_rng(seed)
    return w + 0.05 * rng.standard_normal(w.size)


def test_gradient_matches_oracle():
    dev = _dev()
    w = _perturbed_weights()
    M.mlmc_mlp_set_weights(w)
    w32 = M.mlmc_mlp_get_weights().astype(np.float64)
    u, z = _pairs(8192, 11)
    ut = torch.tensor(u, dtype=torch.float32, device=dev)
    zt = torch.tensor(z, dtype=torch.float32, device=dev)
    g = torch.zeros(M.MLMC_MLP_PARAMS, dtype=torch.float32, device=dev)
    loss = M.mlmc_mlp_grad(ut, zt, g)
    torch.cuda.synchronize()
    # the kernels' input map: v = min(u, 1 - u) in binary32 (exact on the grid), t from binary32 operations
    u32 = u.astype(np.float32).astype(np.float64)
    lo, go = OM.loss_and_grad(w32, O.mlp_feature32(np.minimum(u32, 1.0 - u32)), z.astype(np.float32).astype(np.float64))
    gg = g.cpu().numpy().astype(np.float64)
    assert abs(loss - lo) <= 1e-2 * lo
    # binary16 operands (2^-11 relative) with FP32 accumulation against FP64 backprop: 1e-2 relative
    assert np.linalg.norm(gg - go) <= 1e-2 * np.linalg.norm(go)
    # every block of the layout, not only the largest entries
    for a, b in [(0, 32), (32, 64), (64, 1088), (1088, 1120), (1120, 1152), (1152, 1153)]:
        assert np.linalg.norm(gg[a:b] - go[a:b]) <= 1e-2 * np.linalg.norm(go[a:b]) + 1e-7, (a, b)


def test_forward_matches_oracle():
    dev = _dev()
    w = _perturbed_weights(3)
    M.mlmc_mlp_set_weights(w)
    w32 = M.mlmc_mlp_get_weights().astype(np.float64)
    u = np.concatenate([uniform_grid_sample(100003, 5), [2.0 ** -24, 1 - 2.0 ** -24, 0.25, 0.75]])
    z = torch.empty(u.size, dtype=torch.float32, device=dev)
    M.approx_icdf(torch.tensor(u, dtype=torch.float32, device=dev), z, M.MLMC_ICDF_MLP, M.MLMC_F32)
    torch.cuda.synchronize()
    got = z.cpu().numpy().astype(np.float64)
    ref16 = O.approx_icdf(u, O.RV_MLP16, prec=O.F32, mlp=w32)
    ref64 = O.approx_icdf(u, O.RV_MLP, mlp=w32)
    # the binary16 inference arithmetic, every operation rounded once: bit for bit
    bad = np.flatnonzero(got != ref16)
    assert bad.size == 0, (bad.size, u[bad[:3]], got[bad[:3]], ref16[bad[:3]])
    # and the FP64 network within the binary16 evaluation error (pinned on the oracle side)
    assert np.abs(got - ref64).max() < 4e-3
    # binary16 output: the binary32 value rounded once
    z16 = torch.empty(u.size, dtype=torch.float16, device=dev)
    M.approx_icdf(torch.tensor(u, dtype=torch.float32, device=dev), z16, M.MLMC_ICDF_MLP, M.MLMC_F16)
    torch.cuda.synchronize()
    assert np.array_equal(z16.cpu().numpy().astype(np.float64), O.approx_icdf(u, O.RV_MLP16, prec=O.F16, mlp=w32))


def test_grid_table_equals_direct_evaluation():
    """The level kernels take the network's normals from its values on the
    2^22 grid points v_k = (2k + 1) 2^-24 of v = min(u, 1 - u), tabulated
    when the weights change.  The table must equal the network evaluated
    directly (approx_icdf) and the oracle's binary16 reading at every grid
    point, bit for bit -- after setting weights and after one training step."""
    dev = _dev()
    k = np.arange(1 << 22, dtype=np.float64)
    u = (2.0 * k + 1.0) * 2.0 ** -24
    ut = torch.tensor(u, dtype=torch.float32, device=dev)
    for step in range(2):
        if step == 0:
            M.mlmc_mlp_set_weights(_perturbed_weights(5))
        else:
            uu, zz = _pairs(8192, 3)
            opts = M.mlmc_train_opts(steps=1, batch=4096, lr0=1e-3, lr_min=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                                     seed=5)
            M.mlmc_mlp_train(torch.tensor(uu, dtype=torch.float32, device=dev),
                             torch.tensor(zz, dtype=torch.float32, device=dev), opts)
        z = torch.empty(u.size, dtype=torch.float32, device=dev)
        M.approx_icdf(ut, z, M.MLMC_ICDF_MLP, M.MLMC_F32)
        torch.cuda.synchronize()
        y = M.mlmc_mlp_grid_table()
        assert np.array_equal(-z.cpu().numpy(), y), step      # u_k <= 1/2: Z~ = -y
        w32 = M.mlmc_mlp_get_weights().astype(np.float64)
        ref = O.approx_icdf(u, O.RV_MLP16, prec=O.F32, mlp=w32)
        bad = np.flatnonzero(-y != ref)
        assert bad.size == 0, (step, bad.size, bad[:5])


def _minibatch_indices(n, batch, step, seed):
    ctr = np.zeros((batch, 4), dtype=np.uint32)
    ctr[:, 0] = np.arange(batch, dtype=np.uint32)
    ctr[:, 1] = step
    ctr[:, 3] = 0x4D4C50
    words = O.philox4x32_10(ctr, O.seed_key(seed))
    return ((words[:, 0].astype(np.uint64) * np.uint64(n)) >> np.uint64(32)).astype(np.int64)


def test_one_adam_step_matches_oracle():
    dev = _dev()
    w = _perturbed_weights(9)
    M.mlmc_mlp_set_weights(w)
    w0 = M.mlmc_mlp_get_weights().astype(np.float64)
    n, batch = 50000, 4096
    u, z = _pairs(n, 21)
    ut = torch.tensor(u, dtype=torch.float32, device=dev)
    zt = torch.tensor(z, dtype=torch.float32, device=dev)
    lr = 1e-3
    opts = M.mlmc_train_opts(steps=1, batch=batch, lr0=lr, lr_min=lr, beta1=0.9, beta2=0.999, eps=1e-8, seed=77)
    M.mlmc_mlp_train(ut, zt, opts)
    w1 = M.mlmc_mlp_get_weights().astype(np.float64)
    idx = _minibatch_indices(n, batch, 0, 77)
    u32, z32 = u.astype(np.float32).astype(np.float64), z.astype(np.float32).astype(np.float64)
    _, g = OM.loss_and_grad(w0, O.mlp_feature32(np.minimum(u32[idx], 1.0 - u32[idx])), z32[idx])
    expect, _, _ = OM.adam_step(w0, g, np.zeros_like(g), np.zeros_like(g), 1, lr)
    big = np.abs(g) > 0.02 * np.abs(g).max()
    assert big.sum() > 100
    # the first Adam step moves each weight by ~lr against the sign of its gradient
    assert np.all(np.sign(w1 - w0)[big] == np.sign(expect - w0)[big])
    assert np.allclose((w1 - w0)[big], (expect - w0)[big], rtol=2e-3, atol=1e-7)


@pytest.fixture(scope="module")
def trained():
    dev = _dev()
    M.mlmc_mlp_set_weights(mlp_initial_weights(1234))
    u, z = _pairs(1 << 20, 31)
    ut = torch.tensor(u, dtype=torch.float32, device=dev)
    zt = torch.tensor(z, dtype=torch.float32, device=dev)
    opts = M.mlmc_train_opts(steps=20000, batch=8192, lr0=1e-2, lr_min=1e-5, beta1=0.9, beta2=0.999, eps=1e-8,
                             seed=SEED)
    loss = M.mlmc_mlp_train(ut, zt, opts)
    return M.mlmc_mlp_get_weights().astype(np.float64), loss


def _l2_error_icdf(kind, dev, n=1 << 21):
    u = uniform_grid_sample(n, 41)
    z = torch.empty(n, dtype=torch.float32, device=dev)
    M.approx_icdf(torch.tensor(u, dtype=torch.float32, device=dev), z, kind, M.MLMC_F32)
    torch.cuda.synchronize()
    return float(np.mean((z.cpu().numpy().astype(np.float64) - O.ndtri(u)) ** 2))


def test_trained_network_beats_table(trained):
    dev = _dev()
    w, loss = trained
    M.mlmc_mlp_set_weights(w)
    e_mlp = _l2_error_icdf(M.MLMC_ICDF_MLP, dev)
    e_tab = _l2_error_icdf(M.MLMC_ICDF_TABLE, dev)
    assert abs(e_tab - 4.16e-5) < 0.05e-5
    assert e_mlp < 0.5 * e_tab, (e_mlp, e_tab, loss)


def test_fourway_with_mlp_paths_and_gain(trained, pl_table):
    dev = _dev()
    w, _ = trained
    M.mlmc_mlp_set_weights(w)
    w32 = M.mlmc_mlp_get_weights().astype(np.float64)
    params = M.sde_params(sde=M.MLMC_GBM, payoff=M.MLMC_PAYOFF_CALL, p0=0.05, p1=0.2, K=1.0)
    osde = O.SDE(params.sde, params.payoff, params.p0, params.p1, params.p2, params.x0, params.T, params.K,
                 params.disc)
    # Per path, bar pair binary16 + Kahan with the network: within the
    # workload's 2e-3 (relative to max(1, |P_f|)) of the FP64 oracle (FP64
    # network, FP64 Euler), and bit for bit the oracle's binary16 emulation
    # (binary16 network and Euler).  Hat pair (FP32 + Kahan, exact normals)
    # within 1e-5 of FP64.
    for l, N in ((2, 4001), (6, 2049), (10, 257), (12, 97)):
        out = torch.empty(N * 5, dtype=torch.float32, device=dev)
        M.mlmc_level_paths(1, l, N, M.MLMC_F16, True, M.MLMC_ICDF_MLP, params, SEED, 0, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.float64).reshape(N, 5)
        tag = O.make_tag(O.KIND_FOUR, l)
        ref = O.fourway_paths(l, np.arange(N), O.variant(), O.variant(rv=O.RV_MLP), osde, SEED, tag, mlp=w32)
        emu = O.fourway_paths(l, np.arange(N), O.variant(), O.variant(prec=O.F16, kahan=True, rv=O.RV_MLP16), osde,
                              SEED, tag, mlp=w32)
        scale = np.maximum(1.0, np.abs(ref[:, 0]))
        assert np.all(np.abs(got[:, :2] - ref[:, :2]) <= 1e-5 * scale[:, None]), l
        assert np.all(np.abs(got[:, 2:4] - ref[:, 2:4]) <= 2e-3 * scale[:, None]), l
        assert np.array_equal(got[:, 2:4], emu[:, 2:4]), (l, np.flatnonzero(np.any(got[:, 2:4] != emu[:, 2:4], axis=1)))
    # What the network gains.  Lemma 3.1: the four-way variance is
    # O(delta E|Z - Z~|^2) + O(delta^-1 rho^2).  With FP32 bar paths the first
    # term dominates and the network's smaller E|Z - Z~|^2 shows directly;
    # with binary16 (rho^2 ~ 2.4e-7) the rounding term already dominates at
    # these levels, so the network can only match the table there.
    for l in (2, 4, 6, 8):
        v = {}
        for prec in (M.MLMC_F32, M.MLMC_F16):
            for icdf in (M.MLMC_ICDF_MLP, M.MLMC_ICDF_TABLE):
                v[prec, icdf] = M.mlmc_nested_level(l, 1 << 18, prec, True, icdf, params, SEED).var
        assert v[M.MLMC_F32, M.MLMC_ICDF_MLP] < 0.5 * v[M.MLMC_F32, M.MLMC_ICDF_TABLE], (l, v)
        assert v[M.MLMC_F16, M.MLMC_ICDF_MLP] < 1.05 * v[M.MLMC_F16, M.MLMC_ICDF_TABLE], (l, v)


def test_nested_estimator_with_mlp_is_unbiased(trained):
    """Two-way (MLP) + four-way level means equal the standard estimator's
    level means (both estimate E[P^_l - P^_{l-1}]) within statistical error."""
    _dev()
    w, _ = trained
    M.mlmc_mlp_set_weights(w)
    params = M.sde_params(sde=M.MLMC_GBM, payoff=M.MLMC_PAYOFF_CALL, p0=0.05, p1=0.2, K=1.0)
    for l in (0, 1, 3, 5):
        N = 1 << 20
        a = M.mlmc_level(l, N, M.MLMC_F16, True, M.MLMC_ICDF_MLP, params, SEED)
        b = M.mlmc_nested_level(l, N, M.MLMC_F16, True, M.MLMC_ICDF_MLP, params, SEED)
        c = M.mlmc_level(l, N, M.MLMC_F32, False, M.MLMC_ICDF_EXACT, params, SEED)
        nested = a.mean + b.mean
        se = math.sqrt(a.var / N + b.var / N + c.var / N)
        assert abs(nested - c.mean) < 4.5 * se, (l, nested, c.mean, se)
