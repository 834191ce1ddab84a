"""The 3D leaf evaluation on the tensor cores (tcgen05, TF32 with split operands) against the
same plan on the FP32 FMA pipes and against the FP64 Ewald oracle.

Both paths evaluate the same local expansions at the same targets; the split-TF32 products
carry the accuracy of FP32, so the two results agree to a few FP32 roundings of the local
part (bar: relative L2 difference <= 1e-6 of the potential, 1e-5 of the gradient), and the
tensor-core path holds the oracle bar (eps for the potential, 10 eps for the gradient).  The
split products round each operand twice (about two FP32 roundings per product against one for
an FMA), so the tensor-core path's error against the oracle runs somewhat above the FMA path's
(measured 2.9e-7 against 2.0e-7 on the deep clustered cell at eps 1e-6).
Orders 24 (eps 1e-6) and 16 (eps 1e-3), deep clustered trees, leaves of more than 64 targets
(several row tiles), and a leaf list longer than the persistent grid."""
import numpy as np
import pytest

import workloads as W
from oracle import ewald as E

pytestmark = pytest.mark.gpu


def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_28608_b300 as P
    return P


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


CASES = {
    "triclinic3d_deep": (lambda: W.triclinic3d_clusters(30000, nclusters=8, seed=931), {"n_s": 120}),
    "triclinic3d_small_leaves": (lambda: W.triclinic3d_clusters(20000, nclusters=8, seed=932), {"n_s": 20}),
    "triclinic3d_uniform": (lambda: W.random_neutral(W.lattice_from_lengths_angles(1.0, 1.3, 0.8, 75, 100, 110),
                                                     30000, seed=933), {"n_s": 40}),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("eps", [1e-6, 1e-3])
def test_tensor_core_leaf_evaluation(case, eps):
    P = _cuda()
    make, opts = CASES[case]
    g = make()
    out = {}
    for tc in (True, False):
        plan = P.Plan(g["L"], eps, precision="mixed", tensor_cores=tc, **opts)
        plan.set_sources(g["y"], g["q"])
        out[tc] = plan.eval()
        info = plan.info()
        plan.close()
    assert info["n_proxy"] in (16, 24) and info["pw_eval_targets"] > 0  # leaves were evaluated
    dp, dg = rel(out[True][0], out[False][0]), rel(out[True][1], out[False][1])
    rng = np.random.default_rng(5)
    idx = np.sort(rng.choice(len(g["q"]), 96, replace=False))
    pref, gref = E.ewald(g["L"], g["y"], g["q"], x=g["y"][idx], self_idx=idx)
    ep, eg = rel(out[True][0][idx], pref), rel(out[True][1][idx], gref)
    fp, fg = rel(out[False][0][idx], pref), rel(out[False][1][idx], gref)
    print(f"{case} eps={eps:g} p={info['n_proxy']} leaf targets={info['pw_eval_targets']}: tc vs fma pot "
          f"{dp:.2e} grad {dg:.2e}; oracle: tc E_pot={ep:.2e} E_grad={eg:.2e}, fma E_pot={fp:.2e} E_grad={fg:.2e}")
    assert np.all(np.isfinite(out[True][0])) and np.all(np.isfinite(out[True][1]))
    assert dp <= 1e-6 and dg <= 1e-5
    assert ep <= eps and eg <= 10 * eps
