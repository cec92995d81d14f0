"""Host logic of bench.py: the kernel launches a step claims (the evaluation kernel, the adjoint
kernel plus the unpadding add, and with the piece pre-sort six kernels per chunk of 2^22 queries
for the value forms, five plus the add for the adjoint) and when the pre-sort applies."""
import os
import sys
import types

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_launches_per_step():
    n = 1 << 24                                        # 4 chunks of 2^22
    assert bench.launches_per_step("value", n, False) == 1
    assert bench.launches_per_step("value_grad", n, False) == 1
    assert bench.launches_per_step("adjoint", n, False) == 2
    assert bench.launches_per_step("value", n, True) == 24
    assert bench.launches_per_step("value_grad", n + 1, True) == 30   # a fifth, ragged chunk
    assert bench.launches_per_step("adjoint", n, True) == 21
    assert bench.launches_per_step("adjoint", n, False, True) == 5


def test_adjoint_bins_apply(monkeypatch):
    # the library's rule for the binned adjoint (wide 3-D stencils, many queries)
    monkeypatch.delenv("INTERP_B300_ADJOINT_BINS", raising=False)
    quintic = types.SimpleNamespace(s=3, n_pieces=1, D=2, lookups_per_query=32.0, dims=(128, 128, 128, 1), halo=2,
                                    n_cosets=2)
    fcc = types.SimpleNamespace(s=3, n_pieces=3, D=2, lookups_per_query=16.0, dims=(128, 128, 128, 1), halo=1,
                                n_cosets=4)
    d4s = types.SimpleNamespace(s=4, n_pieces=6, D=2, lookups_per_query=60.0, dims=(48, 48, 48, 48), halo=2,
                                n_cosets=2)
    assert bench.adjoint_bins_apply(quintic, 1 << 24)
    assert not bench.adjoint_bins_apply(quintic, 1 << 16)
    assert not bench.adjoint_bins_apply(fcc, 1 << 24)
    assert not bench.adjoint_bins_apply(d4s, 1 << 24)
    monkeypatch.setenv("INTERP_B300_ADJOINT_BINS", "1")
    assert bench.adjoint_bins_apply(fcc, 10)


def test_presort_applies(monkeypatch):
    monkeypatch.delenv("INTERP_B300_PRESORT", raising=False)
    on = types.SimpleNamespace(presort=1, n_pieces=14)
    off = types.SimpleNamespace(presort=0, n_pieces=6)
    assert bench.presort_applies(on, 1 << 16) and not bench.presort_applies(on, (1 << 16) - 1)
    assert not bench.presort_applies(off, 1 << 24)
    monkeypatch.setenv("INTERP_B300_PRESORT", "1")
    assert bench.presort_applies(off, 10)
    assert not bench.presort_applies(types.SimpleNamespace(presort=0, n_pieces=1), 1 << 24)
    monkeypatch.setenv("INTERP_B300_PRESORT", "0")
    assert not bench.presort_applies(on, 1 << 24)
