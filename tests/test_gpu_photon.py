"""The photon-consumption kernel (sfchem_photon_update, after the
thermochemical step) against the oracle's, on the GPU-updated state.  The
kernel takes its rate factors in FP32 and its photon bookkeeping in FP64,
so: 1e-6 relative on the surviving and the absorbed photons (each from the
formula that keeps it accurate, in thin and opaque cells alike), and photon
number conserved to FP64 rounding; ragged sizes and the in-place update."""
import numpy as np
import pytest

import inputs
import oracle

pytestmark = pytest.mark.gpu
YR = inputs.YR


def _run(cells, dt, in_place=False):
    import torch
    import paper_2604_21438_gb300 as sf
    s = sf.Solver("mixed")
    d = sf.to_device(cells)
    s.step(d, dt, 100.0)
    n = d["n_H"].numel()
    ab = torch.empty((n, 4), dtype=torch.float64, device="cuda")
    if in_place:
        G0, nE = sf.photon_update(d, dt, G0_out=d["G0"], n_euv_out=d["n_EUV"], absorbed=ab)
    else:
        G0, nE = sf.photon_update(d, dt, absorbed=ab)
    torch.cuda.synchronize()
    s.close()
    out = sf.to_host(d)
    return out, G0.cpu().numpy(), nE.cpu().numpy(), ab.cpu().numpy()


@pytest.mark.parametrize("n", [1, 33, 4097, 65536])
def test_photon_update_matches_oracle(n):
    cells = inputs.cells_uniform(n, seed=5)
    dt = 1e3 * YR
    out, G0, nE, ab = _run(cells, dt)
    # the oracle's photon update on the state the GPU step produced
    upd = dict(cells, y_H2=out["y_H2"], y_e=out["y_e"])
    ref = oracle.photon_update(upd, dt)
    np.testing.assert_allclose(nE, ref["n_EUV"], rtol=1e-6, atol=0)
    np.testing.assert_allclose(G0, ref["G0"], rtol=1e-6, atol=0)
    np.testing.assert_allclose(ab, ref["absorbed"], rtol=1e-6, atol=1e-300)
    np.testing.assert_allclose(nE + ab[:, 0] + ab[:, 1], cells["n_EUV"], rtol=1e-15)
    nF = cells["G0"] * oracle.U_HABING / oracle.HNU_FUV
    np.testing.assert_allclose(G0 * oracle.U_HABING / oracle.HNU_FUV + ab[:, 2] + ab[:, 3], nF, rtol=1e-15)


def test_photon_update_in_place_and_empty():
    import torch
    import paper_2604_21438_gb300 as sf
    cells = inputs.cells_gmc(32, seed=9)
    dt = 1e3 * YR
    a = _run(cells, dt, in_place=False)
    b = _run(cells, dt, in_place=True)
    assert np.array_equal(a[1], b[0]["G0"]) and np.array_equal(a[2], b[0]["n_EUV"])
    d = sf.to_device(inputs.cells_uniform(1, seed=1))
    d = {k: v[:0] for k, v in d.items()}
    sf.photon_update(d, dt)
    torch.cuda.synchronize()
