"""The C ABI library loads without a GPU and exports every function that
include/*.h declares (no compute calls)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built_library():
    """Builds librng_gb300.so (nvcc cross-compiles without a GPU) when it is
    missing or older than its sources, so that a fresh checkout can run the
    CPU suite; an up-to-date build costs only the timestamp checks."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("rng_gb300_build",
                                                  os.path.join(ROOT, "paper_1204_6193_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.build()


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        text = re.sub(r"^\s*typedef[^;]*;", "", text, flags=re.M)  # function-pointer types are not exports
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*([a-z_][a-z0-9_]*)\s*\(",
                             text, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["rng_create", "rng_seed", "rng_skipahead", "rng_generate_u32", "rng_generate_f32",
                 "rng_generate_normal", "ising_sweep", "ising_observables"]:
        assert must in names


def test_library_exports_every_declared_symbol(built_library):
    lib = ctypes.CDLL(built_library)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_without_gpu():
    import paper_1204_6193_gb300 as R
    assert R.rng_strerror(R.RNG_OK) == "ok"
    assert "invalid" in R.rng_strerror(R.RNG_EINVAL)


def test_normal_build_reports_no_bounds_checks_without_gpu():
    # the status query of the bounds-check build; the normal build has no
    # checks and says so before touching a device
    import paper_1204_6193_gb300 as R
    if os.environ.get("RNG_GB300_LIBRARY"):
        pytest.skip("another build of the library is loaded")
    with pytest.raises(R.RngError) as e:
        R.rng_debug_bounds_status()
    assert e.value.status == R.RNG_EUNSUPPORTED
