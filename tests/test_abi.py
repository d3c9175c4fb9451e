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


def test_build_targets_sm103a_only():
    """Every translation unit is compiled for sm_103a alone (the GPU tests read the
    architecture of the loaded code back through musr_binary_version)."""
    from paper_1509_07685_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_binary_version_without_gpu_reports_error(lib):
    from conftest import cuda_available
    if cuda_available():
        pytest.skip("a GPU is present")
    from paper_1509_07685_gb300 import binding
    st, _ = binding.musr_binary_version(0)
    assert st == binding.MUSR_EINVAL


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
