"""The C ABI library builds, loads and exports every symbol include/infft.h declares;
argument checks that need no GPU."""
import os
import re

import pytest

import __graft_entry__
import paper_1811_05335_gb300 as g
from paper_1811_05335_gb300 import build as B

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "infft.h")


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:infft_status|int64_t|int32_t|const char\s*\*)\s*(\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_method_calls():
    names = declared_functions()
    for must in ("infft_plan", "infft_precompute", "infft_apply", "nfft_apply", "plan_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol():
    lib = g.library()
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) == set(g.EXPORTED_SYMBOLS)


def test_library_is_sm103a_and_in_tree():
    assert B.lib_path().startswith(os.path.dirname(os.path.dirname(HEADER)))
    assert "arch=compute_103a,code=sm_103a" in B.ARCH


def test_version_and_counter():
    assert "sm_103a" in g.infft_version()
    assert g.infft_launch_count() >= 0


@pytest.mark.parametrize("args,code", [
    ((63, 128, 2.0, 4), 1),            # M odd
    ((0, 128, 2.0, 4), 1),             # M too small
    ((64, 0, 2.0, 4), 1),              # N < 1
    ((64, 128, 0.5, 4), 1),            # sigma < 1
    ((64, 128, 1.01, 4), 1),           # sigma M not an integer
    ((66, 128, 1.5, 4), 1),            # sigma M = 99 odd
    ((64, 128, 2.0, 0), 1),            # m < 1
    ((4, 128, 1.0, 2), 1),             # 2m >= M_sigma
    ((64, 2 ** 30, 2.0, 4), 1),        # N (2m+1) >= 2^31
    ((1000, 4000, 1.5, 4), 5),         # M_sigma = 1500 not a power of two, sigma != 2
    ((8194, 20000, 2.0, 4), 5),        # M_sigma = 16388 not a power of two, M above 8192
])
def test_invalid_sizes(args, code):
    with pytest.raises(g.InfftError) as ei:
        g.infft_plan_create(*args)
    assert ei.value.code == code


def test_invalid_kernel_and_tau():
    with pytest.raises(g.InfftError) as ei:
        g.infft_plan_create(64, 128, 2.0, 4, kernel=7)
    assert ei.value.code == 1
    for tau in (-1.0, 1.0, float("nan")):
        with pytest.raises(g.InfftError):
            g.infft_plan_create(64, 128, 2.0, 4, tau=tau)


def test_invalid_ansatz():
    with pytest.raises(g.InfftError) as ei:
        g.infft_plan_create_ansatz(64, 32, 2.0, 4, ansatz=3)
    assert ei.value.code == 1                      # EINVAL: no such optimisation
    with pytest.raises(g.InfftError) as ei:
        g.infft_plan_create_ansatz(256, 32, 2.0, 9, ansatz="under")
    assert ei.value.code == 5                      # EUNSUPPORTED: 2m+1 = 19 > 17 in the underdetermined case
    with pytest.raises(g.InfftError) as ei:
        g.infft_plan_create_ansatz(48, 32, 2.0, 4, ansatz="under")
    assert ei.value.code == 5                      # M_sigma = 96 not a power of two


def test_null_plan_calls():
    lib = g.library()
    assert lib.plan_destroy(None) == 0
    assert lib.infft_precompute(None, None) == 1
    assert lib.infft_apply(None, None, None, None) == 1
    assert b"NULL" in lib.infft_last_error()
    assert lib.infft_set_nodes(None, None, None) == 1
    assert lib.infft_get_info(None, None) == 1
