"""2-bit packed states on the GPU.

  * jwf_pack_states / jwf_unpack_states equal the oracle's definition of the
    format for ragged lengths, aligned and unaligned buffers;
  * a run loaded from packed initial states equals the oracle's trajectory,
    and its packed history (jwf_step_record_packed) equals the oracle's
    states packed, step by step, for the resident kernels (grids whose rows
    fill whole 32-cell words, and ragged grids whose words share bytes), the
    tiled kernel and the plain one;
  * jwf_get_state_packed equals the packed current state.
"""
import numpy as np
import pytest
import torch

from oracle import discrete
from paper_2512_06102_gb300 import jwf, scenarios
from tests.gpu_util import make_sim, oracle_tables, require_gpu, to

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [1, 3, 4, 15, 16, 17, 1000, 65536 + 7])
@pytest.mark.parametrize("shift", [0, 1])
def test_pack_unpack(n, shift):
    require_gpu()
    rng = np.random.default_rng(n)
    F = rng.integers(0, 4, size=n).astype(np.uint8)
    # shift 1: both buffers start one byte past an aligned address
    src = torch.zeros(n + shift, dtype=torch.uint8, device="cuda")
    src[shift:] = to(F)
    out = torch.zeros(jwf.packed_size(n) + shift, dtype=torch.uint8, device="cuda")
    jwf.pack_states(src[shift:], out=out[shift:])
    ref = discrete.pack_states(F)
    got = out[shift:].cpu().numpy()
    np.testing.assert_array_equal(got[:ref.size], ref)
    assert jwf.packed_size(n) % 16 == 0 and jwf.packed_size(n) >= ref.size
    back = torch.zeros(n + shift, dtype=torch.uint8, device="cuda")
    jwf.unpack_states(out[shift:], n, out=back[shift:])
    np.testing.assert_array_equal(back[shift:].cpu().numpy(), F)


@pytest.mark.parametrize("kernel,shape,N", [
    (jwf.KERNEL_RESIDENT, (64, 96), 4),      # rows of whole words: plain stores
    (jwf.KERNEL_RESIDENT, (37, 45), 5),      # words share bytes: OR into a zeroed row
    (jwf.KERNEL_TILED, (150, 300), 2),
    (jwf.KERNEL_PLAIN, (33, 20), 3),
])
def test_packed_load_and_history_match_oracle(kernel, shape, N):
    require_gpu()
    k = 16
    scn = scenarios.make_scenario(shape[0], shape[1], N=N, seed=61)
    drops = scenarios.drops(k, scn.H, scn.W, seed=6)
    q32 = oracle_tables(scn)[0]
    sim = make_sim(scn, seed=9)
    sim.set_probs(to(q32))
    sim.set_kernel(kernel)
    sim.load_state_packed(to(discrete.pack_states(scn.F0)))
    rows = jwf.packed_size(sim.cells)
    hist = torch.full((k, rows), 0xA5, dtype=torch.uint8, device="cuda")    # stale bytes must be overwritten
    burning, burnt, done = sim.step(k, to(drops), history=hist, packed=True)
    h = hist.cpu().numpy()
    last = sim.state_packed().cpu().numpy()
    full = sim.state().cpu().numpy()
    sim.close()
    ro = discrete.Rollout(scn.H, scn.W, scn.F0, q32, scn.params.p_continue, seed=9)
    nb = (ro.F.size + 3) // 4
    for t in range(k):
        ro.step(1, np.ascontiguousarray(drops[t:t + 1]))
        np.testing.assert_array_equal(h[t, :nb], discrete.pack_states(ro.F), err_msg=f"step {t}")
    np.testing.assert_array_equal(full, ro.F)
    np.testing.assert_array_equal(last[:nb], discrete.pack_states(ro.F))
