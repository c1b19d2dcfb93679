"""ar_unfold_noalloc's argument checks, on the CPU (they run before any CUDA call).

The checks are the ones ar_load_pattern and ar_unfold make (shared code in the library), plus
the limits of the fixed scratch array. Failures are reported through ar_last_error(NULL),
whose message belongs to the calling thread: a failure on another thread does not rewrite it.
No pointer below is dereferenced: every call is refused before it would touch memory.
"""
import ctypes
import math
import threading

import pytest

from paper_1507_07733_gb300 import binding, synth

FAKE = 1 << 20   # a 16-byte-aligned address that is never dereferenced


def _desc(**over):
    d = synth.make_pattern().desc()
    d.update(over)
    return binding.ar_pattern_desc(**d)


def _event(S=3, N=2048, D=2, fs=200e6, n_refr=1.0):
    return binding.ar_event(S, N, D, -1, fs, n_refr, FAKE, FAKE, FAKE, FAKE, None)


def _outputs():
    o = binding.ar_outputs()
    for name, _ in binding.ar_outputs._fields_:
        if name not in ("peak_time_fine_ns", "snr"):
            setattr(o, name, FAKE)
    return o


def _call(desc, ev, out):
    L = binding.load()
    st = L.ar_unfold_noalloc(ctypes.byref(desc), ctypes.c_void_p(FAKE), ctypes.byref(ev), ctypes.byref(out),
                             ctypes.c_void_p(0))
    return st, L.ar_last_error(None).decode()


@pytest.mark.parametrize("field,value,words", [
    ("az0_rad", math.nan, "finite"), ("zen0_rad", math.inf, "finite"), ("f0_hz", math.nan, "finite"),
    ("df_hz", -1.0, "positive"), ("n_freq", 1, "out of range"), ("daz_rad", 0.1, "2 pi")])
def test_bad_descriptors_are_refused_as_ar_load_pattern_refuses_them(field, value, words):
    st, msg = _call(_desc(**{field: value}), _event(), _outputs())
    assert st == 1 and words in msg


@pytest.mark.parametrize("kw,words", [
    (dict(n_refr=-1.0), "refractive_index"), (dict(n_refr=math.inf), "refractive_index"),
    (dict(S=0), "n_stations"), (dict(D=0), "n_dirs"), (dict(fs=-5.0), "fs_hz"),
    (dict(S=241, N=4096, D=1), "983040"), (dict(D=4097), "4096")])
def test_bad_events_are_refused(kw, words):
    st, msg = _call(_desc(), _event(**kw), _outputs())
    assert st == 1 and words in msg, msg


def test_missing_outputs_are_refused():
    out = _outputs()
    out.status = None
    st, msg = _call(_desc(), _event(), out)
    assert st == 1 and "status" in msg


def test_the_message_of_a_failure_belongs_to_the_calling_thread():
    barrier = threading.Barrier(2)
    seen = {}

    def worker(name, kw):
        _call(_desc(), _event(**kw), _outputs())        # this thread's failure
        barrier.wait()                                   # the other thread fails meanwhile
        barrier.wait()
        seen[name] = binding.load().ar_last_error(None).decode()

    a = threading.Thread(target=worker, args=("a", dict(n_refr=-1.0)))
    b = threading.Thread(target=worker, args=("b", dict(S=241, N=4096, D=1)))
    a.start(); b.start(); a.join(); b.join()
    assert "refractive_index" in seen["a"] and "983040" not in seen["a"]
    assert "983040" in seen["b"] and "refractive_index" not in seen["b"]
