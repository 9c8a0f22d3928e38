"""The differentiable path: DiagramFn's backward (the dms_backward kernel)
against (1) the reference gradient built from the oracle's pairs in float64
(relative error <= 1e-6) and (2) float64 central finite differences of the
loss with a step below half the smallest gap between field values, so that
the order -- hence every pair -- is the same at f +- h (relative error
<= 1e-3)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2505_21266_gb300 as dms
from paper_2505_21266_gb300 import fields

THRESH = 0.05


def generic_field(n, seed):
    """A Gaussian mixture plus U[0, 1e-4) noise with all values distinct (the
    differentiable workload's recipe), re-drawn until the values are distinct."""
    for s in range(seed, seed + 50):
        f = fields.gaussian_mixture((n, n, n), 32, (0.05, 0.2), 1e-4, s).numpy()
        if len(np.unique(f)) == f.size:
            return f
    raise RuntimeError("no generic field found")


def loss64(f64, pairs):
    """The loss in float64 for a fixed set of (birth_vtx, death_vtx) pairs."""
    b = f64[pairs[:, 0]]
    d = f64[pairs[:, 1]]
    p = d - b
    keep = p < THRESH
    return float((p[keep] ** 2).sum())


def oracle_pairs(f):
    r = oracle.run(f)
    out = []
    for which in (oracle.D0, oracle.D2):
        a = r.get(which)
        out.append(np.stack([a["birth_vtx"].astype(np.int64), a["death_vtx"].astype(np.int64)], 1))
    return np.concatenate(out)


def reference_gradient(f, pairs):
    f64 = f.astype(np.float64).ravel()
    g = np.zeros(f.size, dtype=np.float64)
    p = f64[pairs[:, 1]] - f64[pairs[:, 0]]
    keep = p < THRESH
    np.add.at(g, pairs[keep, 0], -2.0 * p[keep])
    np.add.at(g, pairs[keep, 1], 2.0 * p[keep])
    return g.reshape(f.shape)


def gpu_gradient(f):
    x = torch.from_numpy(f).cuda().requires_grad_(True)
    loss = dms.topological_loss(x, THRESH)
    loss.backward()
    return float(loss.item()), x.grad.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("n", [16, 24])
def test_backward_matches_oracle_reference(n):
    f = generic_field(n, 3)
    pairs = oracle_pairs(f)
    ref = reference_gradient(f, pairs)
    loss, g = gpu_gradient(f)
    assert abs(loss - loss64(f.astype(np.float64).ravel(), pairs)) <= 1e-5 * max(1.0, loss)
    scale = np.abs(ref).max()
    assert scale > 0
    assert np.abs(g - ref).max() / scale <= 1e-6


def test_backward_matches_central_differences():
    f = generic_field(24, 11)
    f64 = f.astype(np.float64).ravel()
    gap = np.diff(np.sort(f64)).min()
    h = 0.25 * gap
    pairs = oracle_pairs(f)  # unchanged at f +- h: the order does not move
    _, g = gpu_gradient(f)
    g = g.ravel()
    carriers = np.unique(pairs)
    rng = np.random.default_rng(0)
    sample = np.unique(np.concatenate([carriers[rng.permutation(len(carriers))[:150]],
                                       rng.integers(0, f.size, 50)]))
    fd = np.empty(len(sample))
    for k, v in enumerate(sample):
        fp = f64.copy()
        fp[v] += h
        fm = f64.copy()
        fm[v] -= h
        fd[k] = (loss64(fp, pairs) - loss64(fm, pairs)) / (2 * h)
    scale = np.abs(fd).max()
    assert scale > 0
    assert np.abs(g[sample] - fd).max() / scale <= 1e-3


def test_gradient_descent_simplifies():
    """A few gradient steps on the loss shrink it (the diagram is recomputed
    at every step).  Ties are allowed here: they fall to the vertex offset."""
    f = fields.gaussian_mixture((32, 32, 32), 32, (0.05, 0.2), 1e-4, 5).cuda()
    losses = []
    for _ in range(5):
        x = f.clone().requires_grad_(True)
        loss = dms.topological_loss(x, THRESH)
        loss.backward()
        losses.append(float(loss.item()))
        f = (x - 1e-2 * x.grad).detach()
    assert losses[-1] < losses[0]


def test_backward_kernel_scatter():
    """dms_backward on hand-made pairs: accumulation onto shared carriers and
    no death term for the essential class."""
    rec = np.zeros(3, dtype=dms.PAIR_DTYPE)
    rec["birth_vtx"] = [0, 5, 2]
    rec["death_vtx"] = [5, 5, 0]
    rec["death_id"] = [10, 11, -1]
    pairs = torch.from_numpy(rec.view(np.uint8).reshape(3, 32)).cuda()
    g = torch.tensor([[1.0, 2.0], [3.0, 4.0], [5.0, 6.0]], device="cuda")
    grad = torch.zeros((2, 2, 2), device="cuda")
    dms.backward(pairs, g, grad)
    expect = np.zeros(8)
    expect[0] += 1.0
    expect[5] += 2.0 + 3.0 + 4.0
    expect[2] += 5.0
    assert np.array_equal(grad.cpu().numpy().ravel(), expect)


def test_descent_loop_at_128_cubed():
    """The differentiable workload: a 128^3 mixture of 32 Gaussians plus
    U[0, 1e-4), 100 gradient-descent steps at lr 1e-2 on the topological
    loss, the diagram recomputed at every step.  The loss must fall well
    below its start, and every step's loss must be finite."""
    f = fields.config4(0, "cuda")
    losses = []
    for _ in range(100):
        x = f.clone().requires_grad_(True)
        loss = dms.topological_loss(x, THRESH)
        loss.backward()
        losses.append(float(loss.item()))
        f = (x - 1e-2 * x.grad).detach()
    assert all(np.isfinite(losses))
    assert losses[0] > 0
    assert losses[-1] < 0.5 * losses[0]
