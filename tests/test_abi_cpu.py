"""Library build + C-ABI surface checks that need no GPU."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "logan.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(logan_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def built():
    from paper_2002_05200_gb300 import build
    return build.build()


def test_every_declared_symbol_is_exported(built):
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (logan_[a-z_0-9]+)\b", out))
    declared = _declared()
    assert declared, "no declarations parsed"
    missing = [s for s in declared if s not in exported]
    assert not missing, missing
    from paper_2002_05200_gb300 import logan
    assert set(logan.EXPORTED) <= set(declared)


def test_host_only_entry_points(built):
    from paper_2002_05200_gb300 import logan
    assert "sm_103a" in logan.version()
    assert logan.strerror(logan.EINVAL).startswith("invalid")
    assert logan.strerror(logan.ERANGE)
    n = logan.num_levels()
    assert n == 8
    prev = 0
    for k in range(n):
        w, t = logan.level_info(k)
        assert w > prev and t in (8, 16, 32, 128, 512)
        prev = w
    with pytest.raises(logan.LoganError):
        logan.level_info(n)


def test_ctx_create_without_gpu_fails_cleanly(built):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is visible")
    from paper_2002_05200_gb300 import logan
    with pytest.raises(logan.LoganError) as e:
        logan.Context(0)
    assert e.value.code == logan.ECUDA


def test_null_argument_checks(built):
    from paper_2002_05200_gb300 import logan
    L = logan.lib()
    assert L.logan_ctx_create(None, 0, None) == logan.EINVAL
    assert L.logan_set_option(None, 1, 0) == logan.EINVAL
    assert L.logan_extend_batch(None, None, None, None, 0, 1, -1, -1, 5, None, None, 0, None,
                                None) == logan.EINVAL
