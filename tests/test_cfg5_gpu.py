"""The large nonsymmetric workload: planted spectrum l ~ U[-0.95, 0.95] plus a
rank-32 nonsymmetric term of 2-norm 0.01, k = 3375 by radix 15, split-FP16.

No closed form exists for the perturbed matrix, so results are checked on
probe vectors X (64 N(0,1) columns):
  * at n = 2048, against the oracle's Horner recursion s <- x + A s run on the
    probes (the definition, Eq. neumann); for this spectrum E^[3](A) of
    Lemma 5.7 is ~1e-16, so S_k X is also the radix-15 framework value;
  * at n = 16384 (the full size), through the telescoping property
    (I - A) S_k X = X - A^k X with A^k X ~ 0.95^3375 ~ 0: the relative residual
    || (I - A)(S X) - X || / || X || is bounded by ||I - A|| times the error of S.
"""

import pytest

from oracle import closed_form as CF
from workloads import generators as G

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_PROBES = {"split_fp16": 2e-4, "split_bf16": 2e-3}


def _eval(A_np, dtype):
    import paper_2602_11843_gb300 as nm

    p = nm.Plan(A_np.shape[0], 3375, 15, dtype)
    A = torch.tensor(A_np, dtype=torch.float64, device="cuda")
    S = p(A)
    torch.cuda.synchronize()
    return A, S, p.status()


@pytest.mark.parametrize("dtype", ["split_fp16", "split_bf16"])
def test_probe_parity_reduced_size(dtype):
    inp = G.config_inputs(5, n=2048)
    X = inp["probes"]
    ref = CF.horner_probes(inp["A"], X, 3375)
    _, S, st = _eval(inp["A"], dtype)
    assert st == 0
    got = S.cpu().numpy() @ X
    err = CF.rel_fro(got, ref)
    print(f"cfg5 n=2048 {dtype} probe rel err {err:.3e}")
    assert err < TOL_PROBES[dtype]


def test_full_size_telescoping_residual_on_probes():
    inp = G.config_inputs(5)
    A, S, st = _eval(inp["A"], "split_fp16")
    assert st == 0
    X = torch.tensor(inp["probes"], dtype=torch.float64, device="cuda")
    SX = S @ X
    resid = SX - A @ SX - X
    rel = float(torch.linalg.norm(resid) / torch.linalg.norm(X))
    print(f"cfg5 n=16384 split_fp16 telescoping residual {rel:.3e}")
    assert rel < 1e-3
