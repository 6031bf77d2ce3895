"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point that include/spmm_gb300.h declares, and rejects bad
arguments before touching the device."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2311_18141_gb300 import binding
from paper_2311_18141_gb300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "spmm_gb300.h")


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return binding.load_library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char\*|size_t)\s+(spmm_\w+)\s*\(", text,
                                 flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("spmm_csr", "spmm_plan_create", "spmm_csr_transpose", "spmm_sddmm_csr",
                 "spmm_quantize_rows", "spmm_csr_validate"):
        assert must in names
    assert set(names) == set(binding.EXPORTED)


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", binding.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (spmm_\w+)$", out, flags=re.M))
    missing = set(declared_functions()) - exported
    assert not missing, f"not exported: {missing}"
    for name in declared_functions():
        assert hasattr(lib, name)


def test_library_is_sm103a_only(lib):
    # the build passes exactly one -gencode target
    assert libbuild.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_status_strings_and_version(lib):
    assert binding.status_string(0) == "ok"
    assert "misaligned" in binding.status_string(binding.SPMM_ERR_MISALIGNED)
    assert lib.spmm_version() >= 100


def test_host_argument_checks_return_before_device_work(lib):
    i64 = ctypes.c_int64
    # negative sizes
    rc = lib.spmm_csr(None, None, None, 0, None, None, 0, None, 0, None, 0, -1, 4, 4, 0, 1, 1,
                      0.0, None, None, 0, None)
    assert rc == binding.SPMM_ERR_INVALID_ARG
    # unsupported dtype
    rc = lib.spmm_csr(None, None, None, 9, None, None, 0, None, 4, None, 4, 4, 4, 4, 0, 1, 1,
                      0.0, None, None, 0, None)
    assert rc == binding.SPMM_ERR_UNSUPPORTED
    # M == 0 is a no-op
    rc = lib.spmm_csr(None, None, None, 0, None, None, 0, None, 4, None, 4, 0, 4, 4, 0, 1, 1,
                      0.0, None, None, 0, None)
    assert rc == binding.SPMM_OK
    # N not a multiple of the 16-byte vector (F32 needs N % 4 == 0)
    fake = ctypes.c_void_p(256)
    rc = lib.spmm_csr(fake, fake, fake, 0, None, fake, 0, None, 6, fake, 6, 8, 8, 6, 8, 1, 1,
                      0.0, None, fake, 1 << 20, None)
    assert rc == binding.SPMM_ERR_MISALIGNED
    # a B row stride of 2^32 bytes or more (the kernels keep strides in 32 bits)
    rc = lib.spmm_csr(fake, fake, fake, 0, None, fake, 0, None, 1 << 30, fake, 8, 8, 8, 8, 8, 1,
                      1, 0.0, None, fake, 1 << 20, None)
    assert rc == binding.SPMM_ERR_INVALID_ARG
    rc = lib.spmm_csr(fake, fake, fake, 0, None, fake, 0, None, 8, fake, 1 << 30, 8, 8, 8, 8, 1,
                      1, 0.0, None, fake, 1 << 20, None)
    assert rc == binding.SPMM_ERR_INVALID_ARG
    # tile grid that leaves a column block empty
    rc = lib.spmm_csr(fake, fake, fake, 0, None, fake, 0, None, 8, fake, 8, 8, 8, 8, 8, 1, 4,
                      0.0, None, fake, 1 << 20, None)
    assert rc == binding.SPMM_ERR_INVALID_ARG
    # bad tile_rows
    n = ctypes.c_size_t()
    assert lib.spmm_csr_workspace_size(i64(10), i64(10), i64(8), 0, 1, None,
                                       ctypes.byref(n)) == binding.SPMM_ERR_INVALID_ARG
    # quantize: bad dtype and missing scale
    assert lib.spmm_quantize_rows(fake, 4, 4, 4, binding.SPMM_F32, fake, 4, None,
                                  None) == binding.SPMM_ERR_UNSUPPORTED
    assert lib.spmm_quantize_rows(fake, 4, 4, 4, binding.SPMM_E4M3, fake, 4, None,
                                  None) == binding.SPMM_ERR_INVALID_ARG
    # transpose workspace query is pure host arithmetic
    assert binding.spmm_csr_transpose_workspace_size(100, 50, 1000) > 5 * 4 * 1000
    # validate needs a workspace for its status word
    assert lib.spmm_csr_validate(fake, fake, 4, 4, 4, None, 0,
                                 None) == binding.SPMM_ERR_WORKSPACE
    # host pipeline: null handles and plans are rejected, destroy(NULL) is a no-op
    h = ctypes.c_void_p()
    assert lib.spmm_host_pipe_create(ctypes.byref(h), None, 0, 0, 2,
                                     None) == binding.SPMM_ERR_INVALID_ARG
    assert not h.value
    assert lib.spmm_host_pipe_create(None, fake, 0, 0, 2, None) == binding.SPMM_ERR_INVALID_ARG
    assert lib.spmm_host_pipe_create(ctypes.byref(h), fake, 0, 0, 0,
                                     None) == binding.SPMM_ERR_INVALID_ARG
    assert lib.spmm_host_pipe_create(ctypes.byref(h), fake, 7, 0, 2,
                                     None) == binding.SPMM_ERR_UNSUPPORTED
    assert lib.spmm_host_pipe_create(ctypes.byref(h), fake, 0, binding.SPMM_E4M3, 2,
                                     None) == binding.SPMM_ERR_UNSUPPORTED
    assert lib.spmm_host_pipe_submit(None, fake, fake, fake, fake,
                                     fake) == binding.SPMM_ERR_INVALID_ARG
    assert lib.spmm_host_pipe_wait(None) == binding.SPMM_ERR_INVALID_ARG
    assert lib.spmm_host_pipe_destroy(None) == binding.SPMM_OK
    assert lib.spmm_plan_get_boundaries(None, None, None, None) == binding.SPMM_ERR_INVALID_ARG
    # bounded-wait self-test: workspace and limit are checked on the host
    assert lib.spmm_selftest_wait_timeout(None, 0, 1024, None) == binding.SPMM_ERR_WORKSPACE
    assert lib.spmm_selftest_wait_timeout(fake, 8, 1024, None) == binding.SPMM_ERR_WORKSPACE
    assert lib.spmm_selftest_wait_timeout(fake, 256, 0, None) == binding.SPMM_ERR_INVALID_ARG
    assert lib.spmm_selftest_wait_timeout(fake, 256, (1 << 31) + 1,
                                          None) == binding.SPMM_ERR_INVALID_ARG


def test_workspace_size_grows_with_problem(lib):
    small = binding.spmm_csr_workspace_size(1000, 10000, 32, 1, 1)
    big = binding.spmm_csr_workspace_size(100000, 1000000, 128, 16, 4)
    assert 0 < small < big
