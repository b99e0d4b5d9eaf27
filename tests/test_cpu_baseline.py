"""The multithreaded CPU baseline (oracle/cpu_mt.cpp: Algorithm 2's count / scan / fill
with a per-row sort on all host threads) gives the oracle's permutation bit for bit.
CPU only; it is measurement infrastructure, never part of the library."""
import numpy as np
import pytest

import oracle
from oracle import cpu_mt
from pins import rand_csr, same_csr


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_cpu_mt_equals_oracle(seed):
    rng = np.random.default_rng(seed)
    m, n = 300 + seed * 17, 250 + seed * 31
    A, _, _ = rand_csr(oracle, rng, m, n, 0.05, dtype=np.float32)
    p, q = rng.permutation(m), rng.permutation(n)
    rp, ci, vv = cpu_mt.permute(m, n, A.rowptr, A.colidx, A.values, p, q)
    same_csr(oracle.CSR.of(m, n, rp, ci, vv), oracle.permute(A, p, q), f"cpu_mt seed {seed}")


def test_cpu_mt_symmetric_and_rejects():
    rng = np.random.default_rng(9)
    A, _, _ = rand_csr(oracle, rng, 120, 120, 0.1, dtype=np.float32)
    p = rng.permutation(120)
    rp, ci, vv = cpu_mt.permute(120, 120, A.rowptr, A.colidx, A.values, p)  # q = p: P A P^T
    same_csr(oracle.CSR.of(120, 120, rp, ci, vv), oracle.permute(A, p, p), "cpu_mt P A P^T")
    with pytest.raises(ValueError):
        cpu_mt.permute(120, 120, A.rowptr, A.colidx, A.values, np.zeros(120, np.int64))
    assert cpu_mt.threads() >= 1
