"""Guard bands around every output buffer of the GPU tests (a stand-in for a memory checker).

Each output tensor that ``binding.alloc_outputs`` hands out during a GPU test is placed in the
middle of a larger buffer whose GUARD bytes before and after it are filled with a known byte
pattern. After the test the bands are compared with the pattern: a kernel or a copy that
writes outside the output it was given (a wrong pair index, a stride, a staging size) changes
them and fails the test. Device outputs and host (pinned) outputs alike, so the copies of the
server and of the host-buffer entry point are covered as well as the kernels.
"""
import numpy as np

GUARD = 16 << 10          # bytes before and after each output
PATTERN = 0xA5            # fill byte of the bands
ALIGN = 256               # the output starts 256-byte aligned inside its buffer


class GuardRegistry:
    def __init__(self):
        self.buffers = []   # (name, raw uint8 buffer, start, nbytes)

    def empty(self, shape, dtype, name, **kw):
        import torch
        nbytes = int(np.prod(shape)) * torch.empty((), dtype=dtype).element_size()
        raw = torch.empty(GUARD + nbytes + GUARD + ALIGN, dtype=torch.uint8, **kw)
        raw.fill_(PATTERN)
        start = GUARD + (-(raw.data_ptr() + GUARD) % ALIGN)
        view = raw[start:start + nbytes].view(dtype).view(shape)
        self.buffers.append((name, raw, start, nbytes))
        return view

    def check(self):
        """Every band still holds the pattern; returns the number of buffers checked."""
        import torch
        if torch.cuda.is_available():
            torch.cuda.synchronize()
        for name, raw, start, nbytes in self.buffers:
            lo, hi = raw[:start].cpu().numpy(), raw[start + nbytes:].cpu().numpy()   # the bands only
            bad_lo = np.flatnonzero(lo != PATTERN)
            bad_hi = np.flatnonzero(hi != PATTERN)
            assert bad_lo.size == 0, f"{name}: {bad_lo.size} bytes before the output were written (first at -{start - bad_lo[0]})"
            assert bad_hi.size == 0, f"{name}: {bad_hi.size} bytes after the output were written (first at +{bad_hi[0]})"
        n = len(self.buffers)
        self.buffers.clear()
        return n


def guarded_alloc_outputs(registry, outputs_struct):
    """A drop-in for binding.alloc_outputs whose tensors sit between guard bands."""

    def alloc_outputs(n_dirs, n_stations, n_samples, device="cuda", traces=True, pin_memory=False,
                      fine=False, snr=False):
        import torch
        D, S, N = n_dirs, n_stations, n_samples
        kw = dict(device=device)
        if str(device) == "cpu" and pin_memory:
            kw["pin_memory"] = True
        e = lambda shape, dt, name: registry.empty(shape, dt, name, **kw)
        o = dict(
            efield=e((D, S, 2, N), torch.float32, "efield") if traces else None,
            envelope=e((D, S, N), torch.float32, "envelope") if traces else None,
            peak_idx=e((D, S), torch.int32, "peak_idx"),
            peak_amp=e((D, S), torch.float32, "peak_amp"),
            peak_time_ns=e((D, S), torch.float64, "peak_time_ns"),
            residual_ns=e((D, S), torch.float64, "residual_ns"),
            t0_ns=e((D,), torch.float64, "t0_ns"),
            chi2=e((D,), torch.float64, "chi2"),
            status=e((D, S), torch.int32, "status"),
        )
        if fine:
            o["peak_time_fine_ns"] = e((D, S), torch.float64, "peak_time_fine_ns")
        if snr:
            o["snr"] = e((D, S), torch.float32, "snr")
        return o, outputs_struct(o)

    return alloc_outputs
