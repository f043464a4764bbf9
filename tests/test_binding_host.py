"""The Python binding's buffer checks, on the CPU.

The C calls take bare pointers and fill or read whole fields, so a buffer of
the wrong size, type or layout would be read or written past its end (host
memory, or device memory for the on_device forms). The binding refuses such
buffers before the library sees them. Here the library is a stand-in that
records its calls, and a handle is registered with a 5 x 4 grid.
"""
import types

import numpy as np
import pytest

from paper_1812_05401_gb300 import vplbm as V

NX, NY = 5, 4
H = 0x5000


class StubLib:
    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        def call(*args):
            self.calls.append(name)
            return 0
        return call


@pytest.fixture
def lib(monkeypatch):
    stub = StubLib()
    monkeypatch.setattr(V, "lib", lambda: stub)
    monkeypatch.setitem(V._grids, H, (NX, NY))
    return stub


def test_right_buffers_reach_the_library(lib):
    V.vplbm_populations(H, np.empty((9, NY, NX)))
    V.vplbm_set_populations(H, np.zeros((9, NY, NX), dtype=np.float32))  # converted, then passed
    V.vplbm_moments(H, np.empty((NY, NX)), np.empty((NY, NX)), np.empty((NY, NX)))
    V.vplbm_mask(H, np.empty((NY, NX), dtype=np.uint8))
    V.vplbm_set_mask_and_solid_velocity(H, np.zeros((NY, NX), bool), np.zeros((2, NY, NX)))
    V.vplbm_set_initial_velocity(H, np.zeros((2, NY, NX)))
    V.vplbm_forces_async(H, np.empty((7, 3)))
    assert lib.calls == ["vplbm_populations", "vplbm_set_populations", "vplbm_moments",
                         "vplbm_mask", "vplbm_set_mask_and_solid_velocity",
                         "vplbm_set_initial_velocity", "vplbm_forces_async"]


@pytest.mark.parametrize("call", [
    lambda: V.vplbm_populations(H, np.empty((9, NY, NX - 1))),              # too small
    lambda: V.vplbm_populations(H, np.empty((9, NY, NX), dtype=np.float32)),  # element type
    lambda: V.vplbm_populations(H, np.empty((9, NY, 2 * NX))[:, :, ::2]),   # not contiguous
    lambda: V.vplbm_set_populations(H, np.zeros((9, NY + 1, NX))),
    lambda: V.vplbm_moments(H, np.empty((NY, NX)), np.empty((NY, NX)), np.empty(3)),
    lambda: V.vplbm_mask(H, np.empty((NY, NX), dtype=np.int8)),
    lambda: V.vplbm_set_mask_and_solid_velocity(H, np.zeros((NY, NX + 1))),
    lambda: V.vplbm_set_mask_and_solid_velocity(H, np.zeros((NY, NX)), np.zeros((NY, NX))),
    lambda: V.vplbm_set_initial_velocity(H, np.zeros((NY, NX))),
    lambda: V.vplbm_forces_async(H, np.empty((7, 2))),
    lambda: V.vplbm_forces_async(H, np.empty((7, 3), dtype=np.float32)),
    # a host array where a device buffer is named
    lambda: V.vplbm_populations(H, np.empty((9, NY, NX)), on_device=True),
    lambda: V.vplbm_moments(H, *(np.empty((NY, NX)),) * 3, on_device=True),
])
def test_wrong_buffers_are_refused_before_the_library(lib, call):
    with pytest.raises(ValueError):
        call()
    assert lib.calls == []


def test_read_only_output_is_refused(lib):
    out = np.empty((NY, NX), dtype=np.uint8)
    out.flags.writeable = False
    with pytest.raises(ValueError):
        V.vplbm_mask(H, out)
    assert lib.calls == []


def test_a_state_is_passed_with_its_length(lib, monkeypatch):
    seen = {}

    def load(h, buf, n):
        seen["n"] = n
        return 0
    stub = types.SimpleNamespace(vplbm_load_state=load)
    monkeypatch.setattr(V, "lib", lambda: stub)
    V.vplbm_load_state(H, b"x" * 37)
    assert seen["n"] == 37
    V.vplbm_load_state(H, b"")
    assert seen["n"] == 0  # the library refuses a buffer shorter than a state header


def test_grid_is_forgotten_when_the_solver_is_destroyed(lib):
    V._grids[H + 1] = (3, 3)
    V.vplbm_destroy(H + 1)
    assert H + 1 not in V._grids and lib.calls == ["vplbm_destroy"]
