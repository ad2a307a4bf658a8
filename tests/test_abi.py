"""The C-ABI library loads and exports every entry point include/jwf.h declares.

No compute call is made here (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "jwf.h")).read()
    return sorted(set(re.findall(r"^JWF_API\s+[\w\s\*]+?\b(jwf_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def libjwf():
    from paper_2512_06102_gb300 import build
    build.build()
    import torch  # noqa: F401  (loads the CUDA runtime libjwf links against)
    from paper_2512_06102_gb300 import jwf
    return jwf.lib()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ["jwf_create", "jwf_destroy", "jwf_precompute_probs", "jwf_step", "jwf_apply_action",
                 "jwf_reset", "jwf_step_relaxed_fwd", "jwf_step_relaxed_bwd"]:
        assert name in syms


def test_every_declared_symbol_is_exported(libjwf):
    syms = declared_symbols()
    assert len(syms) >= 20
    for name in syms:
        assert hasattr(libjwf, name), name
    from paper_2512_06102_gb300 import jwf
    assert set(jwf.EXPORTS) == set(syms)


def test_host_side_errors_without_gpu(libjwf):
    # argument validation happens before any CUDA call
    from paper_2512_06102_gb300 import jwf
    assert libjwf.jwf_status_string(0) == b"ok"
    assert libjwf.jwf_status_string(1) == b"invalid argument"
    h = ctypes.c_void_p()
    assert libjwf.jwf_create(None, ctypes.byref(h)) == 1
    cfg = jwf._Config(0, None, None, 11, 0, 0, 1, 0)
    assert libjwf.jwf_create(ctypes.byref(cfg), ctypes.byref(h)) == 1
    assert h.value is None
    assert libjwf.jwf_destroy(None) == 0
    assert libjwf.jwf_step(None, 1, None, None, None, None, None) == 1
    # context-free calls: 2-bit packing sizes and argument checks
    assert libjwf.jwf_packed_size(0) == 0
    assert libjwf.jwf_packed_size(1) == 16            # ceil(1 / 4) rounded up to 16 bytes
    assert libjwf.jwf_packed_size(64) == 16
    assert libjwf.jwf_packed_size(65) == 32
    assert libjwf.jwf_packed_size(-1) == -1
    assert libjwf.jwf_pack_states(-1, None, None, None) == 1
    assert libjwf.jwf_pack_states(5, None, None, None) == 1
    assert libjwf.jwf_unpack_states(5, None, None, None) == 1
    # every context call rejects a null context
    for name, args in [("jwf_set_reorder_steps", (None, 8)), ("jwf_set_tile_copy", (None, 1)),
                       ("jwf_set_tile_copy_wait", (None, 1000, 0)), ("jwf_set_env_priority", (None, None)),
                       ("jwf_load_state_packed", (None, None, None)), ("jwf_get_state_packed", (None, None, None)),
                       ("jwf_check_prob_bound", (None, 0, None, None, None, None, None, None, None, None)),
                       ("jwf_step_masked", (None, 1, None, None, None, None, None))]:
        assert getattr(libjwf, name)(*args) == 1, name
    # context-free mask packing: sizes and argument checks
    assert libjwf.jwf_mask_words(0) == 0
    assert libjwf.jwf_mask_words(1) == 1
    assert libjwf.jwf_mask_words(64) == 2
    assert libjwf.jwf_mask_words(65) == 3
    assert libjwf.jwf_pack_masks(-1, 10, None, None, None) == 1
