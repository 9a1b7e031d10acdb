"""The C ABI library builds for sm_103a, loads and exports every declared symbol (no GPU)."""
import os
import re

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "panther.h")


def _declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"PANTHER_API\s+[\w\s\*]+?\b((?:panther|pantherpp)_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1504_02577_gb300 import build
    build.build()
    import paper_1504_02577_gb300 as pk
    return pk.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 25
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_the_header():
    import paper_1504_02577_gb300 as pk
    assert set(_declared()) == set(pk.SIGNATURES)
    for name in _declared():
        assert callable(getattr(pk, name)), name


def test_sample_size_matches_oracle(lib):
    import paper_1504_02577_gb300 as pk
    for eps, delta, c, T in [(0.01, 0.1, 0.5, 5), (0.05, 0.2, 0.7, 2), (0.003, 0.01, 1.0, 9)]:
        assert pk.panther_sample_size(eps, delta, c, T) == oracle.sample_size(eps, delta, c, T)
    with pytest.raises(pk.PantherError):
        pk.panther_sample_size(0.01, 0.1, 0.5, 1)
    with pytest.raises(pk.PantherError):
        pk.panther_sample_size(1.5, 0.1, 0.5, 5)


def test_create_without_device_is_an_error_not_a_crash(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1504_02577_gb300 as pk
    with pytest.raises(pk.PantherError):
        pk.panther_create(0)


def test_library_targets_sm_103a_only():
    from paper_1504_02577_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
