import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


# ----------------------------------------------------------------- shared helpers

LETTERS = "IXYZ"
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_golden(name):
    """Rows of a golden fixture under tests/golden ('#' starts a comment)."""
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                rows.append(line.split())
    return rows


def parse_strings(strs):
    """List of equal-length letter strings -> (n, x (W,M) u64, z (W,M) u64).

    The leftmost letter is qubit 0; Table I of the paper: I=(0,0), Z=(0,1),
    X=(1,0), Y=(1,1)."""
    from paper_2605_25974_gb300.workloads import pack_bits
    n = len(strs[0])
    m = len(strs)
    xb = np.zeros((m, n), bool)
    zb = np.zeros((m, n), bool)
    for t, s in enumerate(strs):
        for q, ch in enumerate(s):
            xb[t, q] = ch in "XY"
            zb[t, q] = ch in "YZ"
    return n, pack_bits(xb, n), pack_bits(zb, n)


def format_strings(n, x, z):
    from paper_2605_25974_gb300.workloads import unpack_bits
    xb = unpack_bits(np.asarray(x).reshape(-1, np.asarray(x).shape[-1]), n)
    zb = unpack_bits(np.asarray(z).reshape(-1, np.asarray(z).shape[-1]), n)
    out = []
    for t in range(xb.shape[0]):
        out.append("".join("IZXY"[2 * int(a) + int(b)] for a, b in zip(xb[t], zb[t])))
    return out


def keys_as_tuples(x, z):
    """(W,M) x/z words -> list of key tuples (x_0..x_{W-1}, z_0..z_{W-1})."""
    k = np.concatenate([x, z], axis=0).T
    return [tuple(int(v) for v in row) for row in k]


@pytest.fixture(scope="session")
def oracle():
    from oracle import pauli_oracle
    pauli_oracle._load()
    return pauli_oracle
