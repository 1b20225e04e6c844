"""Host-only checks of the C ABI (no GPU needed): the library builds and loads,
exports every entry point include/dsp.h declares, validates arguments before
touching the device, and its pulse sampler agrees with the oracle's own."""
import math
import os
import re

import numpy as np
import pytest

from paper_1607_03062_gb300 import binding as B
from paper_1607_03062_gb300 import build as Bd
from paper_1607_03062_gb300 import workloads as W

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "dsp.h")


@pytest.fixture(scope="module")
def lib():
    Bd.build()
    return B.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dsp_[a-z_]+)\s*\(", text)))


def test_header_declares_what_the_binding_wraps():
    assert declared_functions() == sorted(B.EXPORTS)


def test_every_entry_point_cites_its_passage_or_has_none():
    """Each declaration's comment (the last one before it) cites the paper's
    section or equation that defines the operation, or says that the paper has
    no counterpart; the serving calls sit under a section comment that says so."""
    text = open(HEADER).read()
    serving = text.find("/* Serving:")
    assert serving > 0 and "not in the paper" in text[serving:serving + 200]
    names = []
    for m in re.finditer(r"^(?:dsp_status|int64_t|const char \*)\s*(dsp_\w+)\s*\(", text, re.M):
        name = m.group(1)
        names.append(name)
        before = text[:m.start()]
        comment = before[before.rfind("/*"):]
        cites = re.search(r"Sec\.|Eq\.|no[\s*]+counterpart|not in the paper", comment, re.I)
        assert cites or (name.startswith("dsp_server_") and m.start() > serving), name
    assert sorted(names) == declared_functions()


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_state_bytes(lib):
    assert B.state_bytes(64, 64, "fp64") == 32 * 64 * 64
    assert B.state_bytes(3, 5, "fp32_mixed") == 32 * 15
    assert B.state_bytes(0, 5, "fp64") == -1
    assert B.state_bytes(5, 5, 7) == -1
    assert B.state_bytes(65536, 65536, "fp64") == -1  # more than 2^31 - 1 points


@pytest.mark.parametrize("args", [
    (0, 4, (-1, 1), (-1, 1), 1, 0, 1),          # empty grid
    (4, 4, (1, -1), (-1, 1), 1, 0, 1),          # px_min > px_max
    (4, 4, (-1, float("nan")), (-1, 1), 1, 0, 1),
    (4, 4, (-1, 1), (-1, 1), 2, 0, 1),          # bad precision
    (4, 4, (-1, 1), (-1, 1), 1, 5, 1),          # bad scheme
    (4, 4, (-1, 1), (-1, 1), 1, 0, 0),          # bad valley
])
def test_create_grid_rejects_bad_arguments(lib, args):
    with pytest.raises(B.DSPError) as e:
        B.create_grid(*args)
    assert e.value.code == -1


def test_null_handles_are_rejected(lib):
    for call in (lambda: B.evolve(0, 1), lambda: B.project(0, 0), lambda: B.reduce_density(0)):
        with pytest.raises(B.DSPError) as e:
            call()
        assert e.value.code == -1
    B.destroy_grid(0)  # NULL is fine
    assert B.status_string(-5).startswith("time step")


def test_sampler_rejects_bad_specs(lib):
    with pytest.raises(B.DSPError):
        B.sample_pulse({"kind": "sin2", "E0": 1, "omega": 0.0, "T": 1.0}, 10)
    with pytest.raises(B.DSPError):
        B.sample_pulse({"kind": "sin2", "E0": 1, "omega": 1.0, "T": float("inf")}, 10)
    with pytest.raises(B.DSPError):
        B.sample_pulse(W.sin2_pulse(1.0, 1.55, 5.0), 0)


@pytest.mark.parametrize("spec", [
    W.sin2_pulse(1.0, 1.55, 5.0), W.sin2_pulse(2.5, 0.9, 5.0, eps=0.7),
    W.gauss_pulse(2.0, 1.55, 4.0), W.two_colour_pulse(3.0, 1.55, 10.0, 0.5, math.pi / 3),
    W.const_field_pulse(1.3, 40.0), W.zero_pulse(3.0),
])
def test_sampler_agrees_with_oracle(lib, orc, spec):
    """Two independent pulse evaluators (library C++ and oracle C) must agree."""
    n = 977
    a, ai, ao, dt = B.sample_pulse(spec, n)
    b, bi, bo, dtb = orc.pulse_table(spec, n)
    assert dt == dtb
    scale = max(1.0, np.abs(b).max())
    assert np.abs(a - b).max() <= 4e-15 * scale
    assert np.abs(ai - bi).max() <= 4e-15 * scale and np.abs(ao - bo).max() <= 4e-15 * scale


def test_paper_pulse_closed_form_matches_oracle_quadrature(lib, orc):
    """Library: A_x = -int E_x in closed form; oracle: Gauss-Legendre quadrature."""
    spec = W.paper_pulse()
    a, ai, ao, dt = B.sample_pulse(spec, 4000)
    b, bi, bo, _ = orc.pulse_table(spec, 4000)
    scale = np.abs(b).max()
    assert scale > 0.1
    assert np.abs(a - b).max() <= 1e-12 * scale and abs(ao[0] - bo[0]) <= 1e-12 * scale


def test_gauss_sampler_agrees_with_oracle(lib, orc):
    for spec in (W.sin2_pulse(1.0, 1.55, 5.0, eps=0.3), W.paper_pulse(phi=0.7),
                 W.gauss_pulse(2.0, 1.55, 4.0)):
        a, ai, ao, dt = B.sample_pulse_gauss(spec, 611)
        b, bi, bo, dtb = orc.pulse_table_gauss(spec, 611)
        scale = max(1.0, np.abs(b).max())
        assert dt == dtb and np.abs(a - b).max() <= 1e-12 * scale
