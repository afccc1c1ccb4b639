"""Learned-estimator pipeline: generated pairs agree with the oracle, the
closed form on counts matches the oracle, and the MLP kernels match a plain
PyTorch FP32 reference (BF16 rounding emulated)."""
import numpy as np
import pytest

import oracle
from tests.helpers import assert_close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1910_04658_gb300 import binding as B  # noqa: E402
from paper_1910_04658_gb300 import learned as L  # noqa: E402


@pytest.mark.parametrize("N", [256, 1024])
def test_dense_pairs_agree_with_oracle(N):
    n, d, mc = 120, 100_000, 8 * N
    counts = torch.empty((n, 3), dtype=torch.int32, device="cuda")
    sizes = torch.empty((n, 3), dtype=torch.int32, device="cuda")
    cols = torch.full((n, mc), -1, dtype=torch.int32, device="cuda")
    B.bs_dense_pairs(n, N, d, N // 4, 4 * N, 77, 3, counts, sizes, cols, mc)
    torch.cuda.synchronize()
    c, s, cl = (t.cpu().numpy().view(np.uint32) for t in (counts, sizes, cols))
    rows, rp = [], [0]
    for p in range(n):
        A, Bz, I = (int(v) for v in s[p])
        assert N // 4 <= A <= 4 * N and N // 4 <= Bz <= 4 * N and I <= min(A, Bz)
        cc = cl[p, :A + Bz - I]
        assert len(set(cc.tolist())) == cc.size and cc.max() < d          # distinct columns
        a_set = np.sort(cc[:A])
        b_set = np.sort(np.concatenate([cc[:I], cc[A:]]))
        rows += [a_set, b_set]
    row_ptr = np.zeros(2 * n + 1, np.uint64)
    row_ptr[1:] = np.cumsum([r.size for r in rows])
    col = np.concatenate(rows).astype(np.uint32)
    sk, pc = oracle.sketch(row_ptr, col, d, N, seed=3)
    for p in range(n):
        assert pc[2 * p] == c[p, 0] and pc[2 * p + 1] == c[p, 1]
        assert oracle.counts(sk[2 * p:2 * p + 1], sk[2 * p + 1:2 * p + 2])[0, 0] == c[p, 2]
    ex = oracle.exact_pairs(row_ptr, col, np.arange(0, 2 * n, 2), np.arange(1, 2 * n, 2))
    assert np.allclose(ex, L.exact_similarities(s), rtol=0, atol=1e-12)


def test_closed_form_on_counts_matches_oracle():
    # set pairs of the dense regime drawn on the host (|a|, |b| uniform in
    # [N/4, 4N], overlap uniform in [0, min]); the oracle sketches them and
    # gives the counts, the GPU's closed form runs on those counts
    N, n, d = 1024, 700, 100_000
    rng = np.random.default_rng(5)
    rows = []
    for _ in range(n):
        A, Bz = (int(v) for v in rng.integers(N // 4, 4 * N + 1, 2))
        I = int(rng.integers(0, min(A, Bz) + 1))
        cc = rng.choice(d, A + Bz - I, replace=False).astype(np.uint32)
        rows += [np.sort(cc[:A]), np.sort(np.concatenate([cc[:I], cc[A:]]))]
    row_ptr = np.zeros(2 * n + 1, np.uint64)
    row_ptr[1:] = np.cumsum([r.size for r in rows])
    sk, pc = oracle.sketch(row_ptr, np.concatenate(rows), d, N, seed=0)
    c = np.array([[pc[2 * p], pc[2 * p + 1], oracle.counts(sk[2 * p:2 * p + 1], sk[2 * p + 1:2 * p + 2])[0, 0]]
                  for p in range(n)], np.uint32)
    assert (c[:, 0] > 0.9 * N).any()          # some sketches near saturation
    out = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    B.bs_estimate_counts(torch.from_numpy(c.view(np.int32)).cuda(), n, N, out)
    est = out.cpu().numpy()
    ref = np.array([oracle.estimate(*c[i], N)[:4] for i in range(n)])
    for m in range(4):
        assert_close(est[:, m], ref[:, m], m)


def _torch_forward(params, x, with_bound=False):
    bf = lambda v: v.to(torch.bfloat16).to(torch.float32)
    p = bf(params)
    W1, b1 = p[0:256].view(64, 4), p[256:320]
    W2, b2 = p[320:4416].view(64, 64), p[4416:4480]
    W3, b3 = p[4480:4736].view(4, 64), p[4736:4740]
    gelu = lambda z: torch.nn.functional.gelu(z, approximate="tanh")
    h1 = bf(gelu(bf(x) @ W1.T + b1))
    h2 = bf(gelu(h1 @ W2.T + b2))
    out = h2 @ W3.T + b3
    if not with_bound:
        return out
    # The kernels round the same activations to BF16, but evaluate tanh with
    # another approximation and sum in another order, which can move an
    # activation to a neighbouring BF16 value (one step is at most 2^-7 of
    # it); allowing two such steps on every hidden activation bounds the
    # output difference by 2^-6 |h2| |W3|^T.
    return out, (h2.abs() @ W3.abs().T) * 2.0 ** -6


def test_mlp_inference_matches_torch_reference():
    mlp = L.MLPEstimator(seed=4)
    ps = L.dense_pairs(3000, 256, pair_seed=9)
    got = mlp.estimate(ps).cpu()
    x = torch.empty((ps.n, 4), dtype=torch.float32, device="cuda")
    B.bs_mlp_prepare(ps.counts, None, ps.n, 256, x, None)
    scale = torch.tensor([4 * 256, 8 * 256, 1.0, 1.0])
    base = L.closed_form(ps).cpu()
    # an untrained MLP (zero last layer) is exactly the closed form
    assert torch.allclose(got, base, rtol=1e-6, atol=1e-5)
    # with a random (seeded) last layer: closed form + the network's correction
    g = torch.Generator(device="cuda").manual_seed(12)
    mlp.params[4480:4740] = torch.randn(260, device="cuda", generator=g) * 0.1
    corr, bound = _torch_forward(mlp.params.cpu(), x.cpu(), with_bound=True)
    ref = base + corr * scale
    tol = bound * scale + 1e-5 * ref.abs() + 1e-4
    # both inference kernels: the hidden layer on the tensor cores (default)
    # and every layer on the CUDA cores
    outs = []
    for variant in (B.BS_VARIANT_TC, B.BS_VARIANT_POPC):
        out = torch.empty((ps.n, 4), dtype=torch.float32, device="cuda")
        B.bs_mlp_estimate_ex(mlp.params, ps.counts, ps.n, ps.N, out, variant)
        assert B.bs_get_async_error() == 0
        got = out.cpu()
        err = (got - ref).abs()
        assert bool((err <= tol).all()), (variant, float((err / tol).max()))
        outs.append(got)
    # the two differ in the order of FP32 sums and in the tanh evaluation
    # (hardware approximation vs tanhf), which can move an activation by one
    # BF16 rounding step (2^-8 relative) -- within the reference tolerance
    assert bool(((outs[0] - outs[1]).abs() <= 2 * tol).all())
    assert torch.equal(mlp.estimate(ps).cpu(), outs[0])
    # a ragged last tile and a single sample
    for n in (1, 130):
        sub = L.PairSet(ps.N, ps.counts[:n].contiguous(), ps.sizes[:n].contiguous())
        o = torch.empty((n, 4), dtype=torch.float32, device="cuda")
        B.bs_mlp_estimate_ex(mlp.params, sub.counts, n, sub.N, o, B.BS_VARIANT_TC)
        assert torch.allclose(o.cpu(), outs[0][:n], rtol=1e-6, atol=1e-6 * outs[0].abs().max().item())


def test_mlp_gradient_matches_torch_autograd():
    mlp = L.MLPEstimator(seed=6)
    ps = L.dense_pairs(1000, 1024, pair_seed=11)
    x = torch.empty((ps.n, 4), dtype=torch.float32, device="cuda")
    t = torch.empty((ps.n, 4), dtype=torch.float32, device="cuda")
    B.bs_mlp_prepare(ps.counts, ps.sizes, ps.n, 1024, x, t)
    p0 = mlp.params.clone()
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    B.bs_mlp_train_step(mlp.params, mlp.m, mlp.v, mlp.grad, 1, 0.0, x, t, ps.n, loss)
    torch.cuda.synchronize()
    assert torch.equal(mlp.params, p0)                 # lr = 0 leaves the weights alone
    g_kernel = (mlp.m / 0.1).cpu()                     # first Adam moment = 0.1 * gradient
    # reference: same network, BF16 rounding passed straight through in backward
    ste = lambda v: v + (v.to(torch.bfloat16).to(torch.float32) - v).detach()
    P = p0.cpu().clone().requires_grad_(True)
    p = ste(P)
    W1, b1 = p[0:256].view(64, 4), p[256:320]
    W2, b2 = p[320:4416].view(64, 64), p[4416:4480]
    W3, b3 = p[4480:4736].view(4, 64), p[4736:4740]
    gelu = lambda z: torch.nn.functional.gelu(z, approximate="tanh")
    h1 = ste(gelu(ste(x.cpu()) @ W1.T + b1))
    h2 = ste(gelu(h1 @ W2.T + b2))
    y = h2 @ W3.T + b3
    lref = ((y - t.cpu()) ** 2).mean()
    lref.backward()
    assert abs(loss.item() - lref.item()) <= 1e-4 * abs(lref.item()) + 1e-7
    assert torch.allclose(g_kernel, P.grad, rtol=1e-3, atol=1e-3 * P.grad.abs().max().item())


def test_training_reduces_loss():
    mlp = L.MLPEstimator(seed=1)
    sets = [L.dense_pairs(100_000, 256, pair_seed=21), L.dense_pairs(100_000, 1024, pair_seed=22)]
    hist = mlp.train(sets, epochs=6, batch=2048, lr=3e-3)
    assert hist[-1] < hist[0]
    # the MLP starts as the closed form and learns a correction: on held-out
    # pairs its summed scaled error must not exceed the closed form's
    scale = np.array([4.0, 8.0, 1.0, 1.0])
    for N, seed in ((256, 31), (1024, 32)):
        held = L.dense_pairs(50_000, N, pair_seed=seed)
        exact = L.exact_similarities(held.sizes.cpu().numpy())
        sc = np.array([N, N, 1, 1]) * scale
        mlp_err = L.mse_table(mlp.estimate(held).cpu().numpy(), exact)
        cf_err = L.mse_table(L.closed_form(held).cpu().numpy(), exact)
        tot_mlp = sum(mlp_err[m] / sc[i] ** 2 for i, m in enumerate(L.MEASURES))
        tot_cf = sum(cf_err[m] / sc[i] ** 2 for i, m in enumerate(L.MEASURES))
        assert tot_mlp <= tot_cf, (N, mlp_err, cf_err)
    assert np.isfinite(mlp.estimate(sets[0]).cpu().numpy()).all()
