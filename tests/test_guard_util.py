"""The guard-band checker of the GPU tests (tests/guard_util.py), on host tensors: it passes
when only the outputs are written, and fails on a write just before or just after one."""
import pytest

torch = pytest.importorskip("torch")

from guard_util import GUARD, GuardRegistry, guarded_alloc_outputs  # noqa: E402
from paper_1507_07733_gb300 import binding  # noqa: E402


def _alloc():
    reg = GuardRegistry()
    o, st = guarded_alloc_outputs(reg, binding.outputs_struct)(3, 5, 64, device="cpu", fine=True)
    return reg, o, st


def test_outputs_written_in_full_pass():
    reg, o, st = _alloc()
    for v in o.values():
        if v is not None:
            v.fill_(7)
    assert st.efield == o["efield"].data_ptr() and o["efield"].data_ptr() % 256 == 0
    assert reg.check() == 10


@pytest.mark.parametrize("where", ["before", "after"])
def test_a_write_outside_an_output_fails(where):
    reg, o, _ = _alloc()
    name, raw, start, nbytes = next(b for b in reg.buffers if b[0] == "envelope")
    raw[start - 1 if where == "before" else start + nbytes] = 0
    with pytest.raises(AssertionError, match="envelope"):
        reg.check()


def test_bands_are_the_stated_size():
    reg, o, _ = _alloc()
    for name, raw, start, nbytes in reg.buffers:
        assert start >= GUARD and raw.numel() - start - nbytes >= GUARD
