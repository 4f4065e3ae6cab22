"""The C-ABI library loads and exports every symbol include/pasur.h declares (CPU only: no
compute calls), and the host-only entry points behave."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_2508_06559_gb300 import build as B
from paper_2508_06559_gb300 import pasur as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return P.load()


def test_header_symbols_exported(lib):
    header = open(os.path.join(ROOT, "include", "pasur.h")).read()
    declared = set(re.findall(r"^(?:int|const char \*)\s*(pasur_\w+)\(", header, re.M))
    assert declared == set(P.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name


def test_config_default(lib):
    cfg = P.pasur_config_default()
    assert cfg.variant == 0 and cfg.iters == 1000 and abs(cfg.rm_deadzone - 1e-6) < 1e-12
    assert (cfg.dcfr_alpha, cfg.dcfr_beta, cfg.dcfr_gamma) == (1.5, 0.0, 2.0)


def test_library_deal_matches_oracle(lib):
    # both sides implement the same published generator and the paper's pool rule independently
    for seed in list(range(200)) + [2**63 + 5, 123456789]:
        assert P.pasur_deal(seed).tolist() == O.deal(seed).tolist()


def test_create_without_gpu_fails_loudly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(P.PasurError):
        P.Ctx(0)
