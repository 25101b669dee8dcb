"""The usage example of the design notes, end to end on the GPU, with its
results checked against the oracle: grouping of a Jordan-Wigner-shaped H,
H*H, a Clifford gate list in place and one rotation step."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_usage_example(oracle):
    import torch
    from paper_2605_25974_gb300 import paulib, workloads
    from paper_2605_25974_gb300.build import build
    build()
    torch.cuda.init()
    h = workloads.jw(n=100, m=2000)
    gates = [("h", 3, 0), ("cnot", 3, 7)]
    with paulib.PauliSum.from_arrays(h) as H:
        group, n_groups, offsets, members = paulib.group_commuting(H)
        with paulib.multiply(H, H, "fp64") as HH:
            x, z, c, _ = HH.export()
            paulib.apply_clifford(HH, gates)
            with paulib.rotate(HH, h.x[:, 0], h.z[:, 0], 0.1, 0.0) as step:  # no truncation: exact key set
                assert step.is_canonical
                sx, sz, sc, _ = step.export()
    og, ong = oracle.group_commuting(h.n, h.x, h.z)
    assert n_groups == ong and np.array_equal(group.cpu().numpy(), og)
    ox, oz, oc, oabs, _ = oracle.multiply_canonical(h.n, h.as_tuple(), h.as_tuple())
    assert np.array_equal(x, ox) and np.array_equal(z, oz)
    assert (np.abs(c - oc) <= 2e-12 * oabs).all()
    # the step from the oracle: gates on its own product, then the rotation
    gx, gz, gc = ox, oz, oc
    for gate, q1, q2 in gates:
        gx, gz, gc = oracle.apply_clifford(h.n, (gx, gz, gc), gate, q1, q2)
    rx, rz, rc, rabs, _ = oracle.rotate(h.n, (gx, gz, gc), h.x[:, 0], h.z[:, 0], 0.1, 0.0)
    assert np.array_equal(sx, rx) and np.array_equal(sz, rz)
    # errors of H*H carry through the gates (exact) and the rotation (|cos|,
    # |sin| <= 1): bounded by the product's largest sum of contributions
    assert (np.abs(sc - rc) <= 4e-12 * oabs.max()).all()
