"""CPU checks of the C ABI: the library builds, loads and exports every declared entry point;
calls fail with an error code (never a crash) when no GPU is present."""
import re

import pytest

import __graft_entry__  # noqa: F401  (puts the repo root on sys.path)


def declared_symbols():
    text = open(__graft_entry__.ROOT + "/include/polrt.h").read()
    return re.findall(r"^\s*(?:int|size_t|long long|const char \*)\s*(rt_\w+)\(", text, re.M)


@pytest.fixture(scope="module")
def lib():
    from paper_2302_02733_gb300 import build, polrt

    build.build()
    return polrt.lib()


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), n


def test_error_strings(lib):
    from paper_2302_02733_gb300 import polrt

    for code in (0, -1, -2, -3, -4, -5, -6, -7):
        assert polrt.rt_error_string(code)
    assert "unknown" in polrt.rt_error_string(-99)
    assert polrt.rt_workspace_min_bytes() > 0


def test_null_arguments_are_rejected(lib):
    from paper_2302_02733_gb300 import polrt

    assert lib.rt_destroy(None) == polrt.RT_ERR_INVALID
    assert lib.rt_render(None, 0, None, None) == polrt.RT_ERR_INVALID
    assert lib.rt_set_integrator(None, 0.05, 100) == polrt.RT_ERR_INVALID
    assert lib.rt_render_batch(None, 0, None, 0) == polrt.RT_ERR_INVALID
    assert lib.rt_batch_autotune(None, 0, None, 0, None) == polrt.RT_ERR_INVALID
    assert lib.rt_set_batch_config(None, 0, None) == polrt.RT_ERR_INVALID
    assert lib.rt_render_depths(None, 0, None, None, None) == polrt.RT_ERR_INVALID
    assert lib.rt_last_timeline(None, None, 0, None) == polrt.RT_ERR_INVALID


def test_create_without_gpu_reports_an_error():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2302_02733_gb300 import polrt

    with pytest.raises(polrt.PolrtError):
        polrt.rt_create(0, None)


def test_static_render_limit_matches_the_documented_figure(lib):
    """rt_render_static's pixel limit is derived from the same arena constants as rt_render's
    workspace; the header and the design notes state 13076 pixels."""
    from paper_2302_02733_gb300 import polrt

    assert polrt.rt_render_static_max_pixels() == 13076
    assert "13076 pixels" in open(__graft_entry__.ROOT + "/include/polrt.h").read()
