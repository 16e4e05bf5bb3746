"""The viscosity laws as the viscous kernels evaluate them on the device
(cfd_eval_viscosity), against numpy: the table-driven power law T^omega
(2^(e omega) m_k^omega times a binomial series, FP64 and FP32) over the
table's range, its node points and edges and the fallback beyond it, and
Sutherland's law (Eq. 15)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_15333_gb300 import build
    build.build()


def temperatures(seed):
    rng = np.random.default_rng(seed)
    nodes = np.ldexp(1.0 + np.arange(256) / 256.0, rng.integers(-64, 64, 256))   # table nodes m_k 2^e
    below = np.nextafter(nodes, 0.0)                                             # just below a node
    edges = np.array([2.0 ** -64, np.nextafter(2.0 ** 64, 0.0), 1.0, np.nextafter(1.0, 2.0),
                      np.nextafter(2.0, 0.0), 0.5, 3.0])
    flow = np.linspace(0.05, 20.0, 20001)                                        # temperatures of a flow
    wide = np.exp(rng.uniform(np.log(2.0 ** -64), np.log(2.0 ** 64), 20000))
    return np.concatenate([nodes, below, edges, flow, wide])


@pytest.mark.parametrize("omega", [0.76, 0.5, 1.5, 2.0 / 3.0])
def test_power_law_fp64(omega):
    from paper_2209_15333_gb300 import _lib as L
    T = temperatures(1)
    mu = L.eval_viscosity(T, visc_law=L.POWER, visc_omega=omega, precision=0)
    ref = T ** omega
    rel = np.abs(mu - ref) / ref
    print("omega %.4f: max relative error %.3g (%.2f units of 2^-53)" % (omega, rel.max(), rel.max() / 2.0 ** -53))
    assert rel.max() <= 8 * 2.0 ** -53
    # beyond the tables: exp(omega log T), whose rounded argument costs about
    # |omega log T| units of rounding
    Tf = np.array([1e-30, 2.0 ** -65, 2.0 ** 64, 1e25, 5e-324])
    muf = L.eval_viscosity(Tf, visc_law=L.POWER, visc_omega=omega, precision=0)
    ref = Tf ** omega
    assert np.all(np.abs(muf - ref) <= (8.0 + 2.0 * np.abs(omega * np.log(Tf))) * 2.0 ** -53 * ref)


@pytest.mark.parametrize("omega", [0.76, 1.5])
def test_power_law_fp32(omega):
    from paper_2209_15333_gb300 import _lib as L
    T = temperatures(2)
    T32 = T.astype(np.float32).astype(np.float64)
    # the float tables' range (rounding to float can carry a value to 2^64)
    keep = (T32 >= 2.0 ** -64) & (T32 < 2.0 ** 64)
    T, T32 = T[keep], T32[keep]
    mu = L.eval_viscosity(T, visc_law=L.POWER, visc_omega=omega, precision=1)
    ref = T32 ** omega
    rel = np.abs(mu - ref) / ref
    print("omega %.4f FP32: max relative error %.3g (%.2f units of 2^-24)" % (omega, rel.max(), rel.max() / 2.0 ** -24))
    assert rel.max() <= 8 * 2.0 ** -24
    assert np.all(mu == mu.astype(np.float32))


def test_sutherland_fp64():
    from paper_2209_15333_gb300 import _lib as L
    T = np.linspace(0.05, 20.0, 5001)
    mu = L.eval_viscosity(T, visc_law=L.SUTHERLAND, T_ref=108.1, precision=0)
    s = 110.4 / 108.1
    ref = T ** 1.5 * (1.0 + s) / (T + s)
    assert np.abs(mu - ref).max() <= 8 * 2.0 ** -53 * ref.max()


def test_bad_arguments():
    from paper_2209_15333_gb300 import _lib as L
    with pytest.raises(L.CfdError):
        L.eval_viscosity(np.ones(3), visc_law=7)
