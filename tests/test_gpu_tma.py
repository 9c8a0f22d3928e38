"""Large-field paths: the gradient kernel's two ways of staging the order
field, and the order stage's inverse permutation.  Staging: TMA tile loads
(row pitch a multiple of 16 bytes, order 16-byte aligned) and plain loads
(otherwise).  Both must give the same records, and the TMA path must match
the oracle on grids whose x tiles, y tiles and z chunks all end ragged, so
that every border case of its window fix-up is met.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import record_decode as rd

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2505_21266_gb300 as dms
from paper_2505_21266_gb300 import fields


def _misaligned_copy(order_t):
    """The same order values 4 bytes past a 16-byte boundary (plain loads)."""
    n = order_t.numel()
    buf = torch.empty(n + 4, dtype=torch.uint32, device=order_t.device)
    view = buf[1:1 + n].view(order_t.shape)
    view.copy_(order_t)
    assert view.data_ptr() % 16 == 4
    return view


@pytest.mark.parametrize("shape", [(19, 45, 68), (33, 26, 100), (64, 64, 64), (70, 49, 36)])
@pytest.mark.parametrize("kind", ["mixture", "ties"])
def test_tma_and_plain_staging_agree(shape, kind):
    if kind == "mixture":
        f = fields.gaussian_mixture(shape, 8, (0.05, 0.2), 1e-2, sum(shape)).cuda()
    else:
        f = fields.quantized_noise(shape, 8, sum(shape)).cuda()
    o = dms.order(f)
    assert o.data_ptr() % 16 == 0 and shape[2] % 4 == 0  # the TMA path
    a = dms.gradient(o)
    b = dms.gradient(_misaligned_copy(o))
    torch.cuda.synchronize()
    assert int(a.counts[0]) >= 0
    assert torch.equal(a.desc, b.desc)
    assert torch.equal(a.rec, b.rec)
    assert torch.equal(a.counts, b.counts)


@pytest.mark.parametrize("shape", [(19, 45, 68), (9, 30, 36)])
def test_tma_path_matches_oracle(shape):
    rng = np.random.default_rng(sum(shape))
    for f_np in (rng.random(shape).astype(np.float32),
                 rng.integers(0, 4, size=shape).astype(np.float32),
                 fields.gaussian_mixture(shape, 6, (0.1, 0.3), 1e-3, 1).numpy()):
        nz, ny, nx = shape
        r = oracle.run(f_np)
        o = dms.order(torch.from_numpy(f_np).cuda())
        g = dms.gradient(o)
        pairs, crit = rd.decode(g.desc.cpu().numpy(), g.rec.cpu().numpy(), nx, ny, nz)
        assert np.array_equal(pairs, r.get(oracle.GRAD_PAIRS))
        for d in range(4):
            assert np.array_equal(crit[d], r.crit(d))


@pytest.mark.parametrize("kind", ["quantised", "mixture", "one_byte", "constant"])
def test_order_inverse_permutation_path(kind):
    """Fields of at least 2^25 vertices build order[] from the sorted
    payloads by the bucketed inverse permutation; it must equal the inverse
    of a stable argsort, here on a size whose last slices are partial.
    "one_byte": only one key byte varies (one sort pass, reading the field
    itself); "constant": no pass at all (ties: the identity)."""
    shape = (330, 320, 320)  # 33,792,000 vertices
    if kind == "quantised":
        f = fields.quantized_noise(shape, 64, 5).cuda()
    elif kind == "mixture":
        f = fields.gaussian_mixture(shape, 16, (0.05, 0.2), 1e-2, 5, device="cuda")
    elif kind == "one_byte":  # 1 + j/128: only the top mantissa byte varies
        j = fields.quantized_noise(shape, 128, 6).cuda() * 128.0
        f = 1.0 + j / 128.0
    else:
        f = torch.full(shape, 0.5, dtype=torch.float32, device="cuda")
    o = dms.order(f).reshape(-1).to(torch.int64)
    idx = torch.sort(f.reshape(-1) + 0.0, stable=True).indices
    inv = torch.empty_like(idx)
    inv[idx] = torch.arange(idx.numel(), device=idx.device)
    assert torch.equal(o, inv)
