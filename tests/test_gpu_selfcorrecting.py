"""The self-correcting pairing (Sec. 4.3, Alg. 4, as a fixpoint on the GPU:
dms_diagram_d0d2_selfcorrecting) against the oracle's Alg. 1 on small grids
with ties, signed zeros, noise and mixtures, and against the default
pairing (spanning forest + exact rounds) on the 512^3 quantised-noise
workload and a chain of wells, bit for bit."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import oracle_jobs

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2505_21266_gb300 as dms
from paper_2505_21266_gb300 import fields
from test_gpu_configs import _same_pairs, chain_field
from test_gpu_parity import _fields


@pytest.mark.parametrize("shape,seed", [((23, 37, 41), 1), ((64, 33, 35), 2), ((5, 70, 66), 3)])
def test_selfcorrecting_matches_oracle(shape, seed):
    for name, f_np in _fields(shape, seed).items():
        r = oracle.run(f_np)
        d0, d2, ess = oracle_jobs.sorted_pairs(r)
        g = dms.diagram(torch.from_numpy(np.ascontiguousarray(f_np)).cuda(),
                        pairing="selfcorrecting")
        torch.cuda.synchronize()
        _same_pairs(g.diagrams.numpy("d0"), d0)
        _same_pairs(g.diagrams.numpy("d2"), d2)
        assert g.diagrams.numpy("d0_essential")["birth_id"][0] == ess["birth_id"][0], name


def _both(f):
    o = dms.order(f)
    g = dms.gradient(o)
    c = dms.critical(g)
    a = dms.diagram_d0d2(f, o, g, c, pairing="rounds")
    b = dms.diagram_d0d2(f, o, g, c, pairing="selfcorrecting")
    torch.cuda.synchronize()
    for k in ("d0", "d2", "d0_essential"):
        _same_pairs(a.numpy(k), b.numpy(k))


def test_selfcorrecting_equals_rounds_on_quantised_noise_512():
    _both(fields.config2(0, "cuda"))


def test_selfcorrecting_equals_rounds_on_mixture_256():
    _both(fields.config3(0, "cuda", n=256))


def test_selfcorrecting_on_chains_of_wells():
    for deeper_right in (True, False):
        f_np = chain_field(2000, deeper_right)
        r = oracle.run(f_np)
        d0, _, _ = oracle_jobs.sorted_pairs(r)
        g = dms.diagram(torch.from_numpy(f_np).cuda(), pairing="selfcorrecting")
        torch.cuda.synchronize()
        _same_pairs(g.diagrams.numpy("d0"), d0)
