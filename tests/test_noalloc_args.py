"""Host-side checks of the allocation-free entry point's Python binding: every
malformed argument is rejected before anything reaches the C ABI or the GPU
(the kernel reads rowptr[r + 1] and x[col[e]] without bounds checks)."""
import pytest

torch = pytest.importorskip("torch")

from paper_2405_00814_gb300 import fdtd  # noqa: E402


def _good(n=5, e=9):
    rp = torch.zeros(n + 1, dtype=torch.int32)
    col = torch.zeros(e, dtype=torch.int32)
    w = torch.zeros(e, dtype=torch.float32)
    h = torch.zeros(n, dtype=torch.float32)
    return (rp, col, w), (rp.clone(), col.clone(), w.clone()), h


def test_well_formed_arguments_pass():
    l1, l2, h = _good()
    assert fdtd.check_noalloc_args(l1, l2, h, require_cuda=False) == 5


def test_host_tensors_are_rejected():
    l1, l2, h = _good()
    with pytest.raises(ValueError, match="CUDA"):
        fdtd.check_noalloc_args(l1, l2, h)
    with pytest.raises(ValueError, match="CUDA"):
        fdtd.mp_steps_noalloc(l1, l2, h, 1)


@pytest.mark.parametrize("which,bad", [
    ("h", lambda t: t.double()), ("rowptr", lambda t: t.long()), ("col", lambda t: t.long()),
    ("w", lambda t: t.half()),
])
def test_wrong_dtype(which, bad):
    (r, c, w), l2, h = _good()
    if which == "h":
        h = bad(h)
    elif which == "rowptr":
        r = bad(r)
    elif which == "col":
        c = bad(c)
    else:
        w = bad(w)
    with pytest.raises(ValueError, match="dtype"):
        fdtd.check_noalloc_args((r, c, w), l2, h, require_cuda=False)


def test_non_contiguous():
    (r, c, w), l2, h = _good(e=9)
    w = torch.zeros(18, dtype=torch.float32)[::2]
    with pytest.raises(ValueError, match="contiguous"):
        fdtd.check_noalloc_args((r, c, w), l2, h, require_cuda=False)


def test_rowptr_of_another_graph():
    l1, (r2, c2, w2), h = _good(n=5)
    r2 = torch.zeros(4, dtype=torch.int32)            # a smaller graph's rowptr
    with pytest.raises(ValueError, match="rowptr2"):
        fdtd.check_noalloc_args(l1, (r2, c2, w2), h, require_cuda=False)


def test_weights_and_columns_differ_in_length():
    (r, c, w), l2, h = _good(e=9)
    w = torch.zeros(8, dtype=torch.float32)
    with pytest.raises(ValueError, match="w1"):
        fdtd.check_noalloc_args((r, c, w), l2, h, require_cuda=False)


def test_tensors_on_different_devices():
    (r, c, w), l2, h = _good()
    c = torch.zeros(9, dtype=torch.int32, device="meta")
    with pytest.raises(ValueError, match="col1"):
        fdtd.check_noalloc_args((r, c, w), l2, h, require_cuda=False)


def test_not_a_tensor():
    (r, c, w), l2, h = _good()
    with pytest.raises(TypeError):
        fdtd.check_noalloc_args((r, c.numpy(), w), l2, h, require_cuda=False)
