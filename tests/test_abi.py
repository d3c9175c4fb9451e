"""The C ABI library loads and exports every symbol include/musr.h declares (CPU only:
no compute call is made)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "musr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(musr_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1509_07685_gb300 import binding
    return binding.load()


def test_header_declarations_are_exported(lib):
    from paper_1509_07685_gb300 import binding
    decl = _declared()
    assert decl, "no declarations parsed"
    for name in decl:
        assert hasattr(lib, name), f"{name} declared in musr.h but not exported"
    assert sorted(binding.EXPORTS) == decl


def test_library_is_built_for_sm103a():
    import subprocess
    so = os.path.join(ROOT, "paper_1509_07685_gb300", "libmusr.so")
    out = subprocess.run(["cuobjdump", "--list-elf", so], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    assert "sm_103a" in out.stdout


def test_create_without_gpu_reports_error(lib):
    """Without a GPU, musr_ctx_create returns MUSR_ECUDA (no crash, no fallback)."""
    from conftest import cuda_available
    if cuda_available():
        pytest.skip("a GPU is present")
    from paper_1509_07685_gb300 import binding
    with pytest.raises(binding.MusrError) as e:
        binding.musr_ctx_create(0)
    assert e.value.status == binding.MUSR_ECUDA


def test_server_create_without_gpu_reports_error(lib):
    from conftest import cuda_available
    if cuda_available():
        pytest.skip("a GPU is present")
    from paper_1509_07685_gb300 import binding
    with pytest.raises(binding.MusrError) as e:
        binding.musr_server_create(0, 1 << 30, 4)
    assert e.value.status == binding.MUSR_ECUDA


def test_bounded_wait_check_without_gpu_reports_error(lib):
    from conftest import cuda_available
    if cuda_available():
        pytest.skip("a GPU is present")
    from paper_1509_07685_gb300 import binding
    st, _, _ = binding.musr_check_bounded_wait(0)
    assert st == binding.MUSR_EINVAL
