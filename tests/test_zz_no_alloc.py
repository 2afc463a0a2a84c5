"""The allocation-free message-passing entry point against the context path.

fdtd_mp_steps_noalloc is for callers that cannot allocate device memory (a
host allocator that owns all device memory, a real-time loop that cannot take
cudaMalloc's synchronisation).  It must give the
same node values as fdtd_step_edgelist, the existing literal message-passing
entry point, on the same graph and initial state -- checked on two calls in a
row, since every call reuses the same fixed scratch array.  This file is named
to be collected last.
"""
import numpy as np
import pytest

from paper_2405_00814_gb300 import scenes
from tests._helpers import TOL_FIELD, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _csr(torch, n, src, dst, w):
    order = np.lexsort((src, dst))      # grouped by destination (already, but be explicit)
    src, dst, w = src[order], dst[order], w[order]
    rowptr = np.zeros(n + 1, np.int32)
    np.add.at(rowptr, dst + 1, 1)
    rowptr = np.cumsum(rowptr).astype(np.int32)
    dev = "cuda"
    return (torch.from_numpy(rowptr).to(dev), torch.from_numpy(src.astype(np.int32)).to(dev),
            torch.from_numpy(w.astype(np.float32)).to(dev))


def test_noalloc_matches_edgelist_entry_on_two_calls(torch_cuda):
    torch = torch_cuda
    from paper_2405_00814_gb300 import fdtd
    sc = scenes.ellipse_scene(side=96, nsteps=10, npml=8)
    sc.source = None
    ny, nx = sc.ny, sc.nx
    ez = scenes.random_fields(21, (ny, nx)).astype(np.float32)
    ez[0, :] = 0
    ez[:, 0] = 0
    hx = scenes.random_fields(22, (ny, nx), 1e-3).astype(np.float32)
    hy = scenes.random_fields(23, (ny, nx), 1e-3).astype(np.float32)

    sim = fdtd.Simulation(sc)
    sim.set_field("ez", ez)
    sim.set_field("hx", hx)
    sim.set_field("hy", hy)
    n_nodes, s1, d1, w1 = sim.export_graph(1)
    _, s2, d2, w2 = sim.export_graph(2)
    assert n_nodes <= fdtd.MP_NOALLOC_MAX_NODES
    L1 = _csr(torch, n_nodes, s1, d1, w1)
    L2 = _csr(torch, n_nodes, s2, d2, w2)

    # Prop. 1 numbering: u = i + 3 j nx (Hx), q = 2 i + nx (3 j + 1) (Hy), t = q + 1 (Ez);
    # CPML auxiliary nodes start at zero, like the context's psi arrays
    i = np.arange(nx)[None, :]
    j = np.arange(ny)[:, None]
    t_idx = (2 * i + 1 + nx * (3 * j + 1)).ravel()
    u_idx = (i + 3 * j * nx).ravel()
    q_idx = (2 * i + nx * (3 * j + 1)).ravel()
    h0 = np.zeros(n_nodes, np.float32)
    h0[t_idx], h0[u_idx], h0[q_idx] = ez.ravel(), hx.ravel(), hy.ravel()
    h = torch.from_numpy(h0).cuda()

    for call in range(2):
        fdtd.mp_steps_noalloc(L1, L2, h, 37)
        sim.step_edgelist(37)
        torch.cuda.synchronize()
        hn = h.cpu().numpy()
        ref = {c: sim.get_field(c, (ny, nx)) for c in ("ez", "hx", "hy")}
        for c, idx in (("ez", t_idx), ("hx", u_idx), ("hy", q_idx)):
            e = rel_l2(hn[idx].reshape(ny, nx), ref[c])
            assert e <= TOL_FIELD, (call, c, e)
    sim.close()


def test_noalloc_rejects_oversized_graph(torch_cuda):
    torch = torch_cuda
    from paper_2405_00814_gb300 import fdtd
    n = fdtd.MP_NOALLOC_MAX_NODES + 1
    rp = torch.zeros(n + 1, dtype=torch.int32, device="cuda")   # well-formed, only too large
    col = torch.zeros(1, dtype=torch.int32, device="cuda")
    w = torch.zeros(1, dtype=torch.float32, device="cuda")
    h = torch.zeros(n, dtype=torch.float32, device="cuda")
    with pytest.raises(fdtd.FDTDError) as ei:
        fdtd.mp_steps_noalloc((rp, col, w), (rp, col, w), h, 1)
    assert ei.value.code == fdtd.EINVAL
