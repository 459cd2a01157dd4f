"""CPU-side checks of the C ABI: the library loads without a GPU, exports every
symbol include/seraph.h declares, and the ctypes mirror has the C layout.
No compute call is made here."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_1806_00762_b300 as seraph
from paper_1806_00762_b300 import _capi as C

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "seraph.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(seraph_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported_and_bound():
    names = declared_functions()
    assert "seraph_run" in names and "seraph_graph_from_edges" in names
    lib = C.lib()
    for name in names:
        assert hasattr(lib, name), name
        assert name in C.PROTOTYPES, name


def _c_layout(struct, fields):
    src = f"""
#include <stdio.h>
#include <stddef.h>
#include "seraph.h"
int main(void) {{
  printf("%zu\\n", sizeof({struct}));
  {''.join(f'printf("%zu\\n", offsetof({struct}, {f}));' for f in fields)}
  return 0;
}}"""
    d = os.path.join(ROOT, "_build")
    os.makedirs(d, exist_ok=True)
    c = os.path.join(d, f"layout_{struct}.c")
    exe = c[:-2]
    open(c, "w").write(src)
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    return [int(x) for x in out]


@pytest.mark.parametrize("name,cls", [("seraph_params", C.Params), ("seraph_stats", C.Stats),
                                      ("seraph_graph_info", C.GraphInfo),
                                      ("seraph_batch_params", C.BatchParams),
                                      ("seraph_batch_stats", C.BatchStats),
                                      ("seraph_query", C.Query), ("seraph_trace", C.Trace)])
def test_struct_layout_matches_header(name, cls):
    fields = [f for f, _ in cls._fields_ if not f.startswith("pad")]
    got = _c_layout(name, fields)
    assert got[0] == ctypes.sizeof(cls)
    for f, off in zip(fields, got[1:]):
        assert getattr(cls, f).offset == off, f


def test_params_default_without_gpu():
    p = seraph.default_params("pagerank")
    assert p.algo == C.PAGERANK and p.max_sweeps == 100 and abs(p.damping - 0.85) < 1e-15
    assert p.tol == 1e-7 and p.kahan == 1 and p.verify == 1
    # weak state machine: 0,1,5 attempt, 2,3,4 dormant
    assert p.fsm_skip_mask == 0b011100
    nxt = list(p.fsm_next)
    assert (nxt[0], nxt[1]) == (5, 0) and (nxt[10], nxt[11]) == (3, 0)
    assert (nxt[6], nxt[4], nxt[2]) == (2, 1, 4)


def test_null_arguments_are_rejected_with_message():
    lib = C.lib()
    rc = lib.seraph_run(None, None, None, 0, None)
    assert rc == C.SERAPH_EINVAL
    assert b"null" in lib.seraph_last_error()
    assert lib.seraph_params_default(None, 0) == C.SERAPH_EINVAL


def test_input_module_and_oracle_libraries_load():
    import oracle
    import synth
    synth._dev_lib()
    oracle._L()
    assert hasattr(synth._dev_lib(), "synth_rmat_device")


def test_sched_targets_on_a_handmade_trace():
    """k = smallest number of passes holding >= share of the step's changes;
    priority = log2(1 + first-pass changes) / 24 (host code, no GPU)."""
    import numpy as np
    tr = seraph.TraceBuffer(3)
    tr.gains[0, :4] = [100, 10, 0, 0]     # 110 total: 100/110 < .95 -> k = 2
    tr.gains[1, :3] = [0, 0, 0]           # no change: k = 1
    tr.gains[2, :16] = 1                  # uniform: need 16 * .95 -> 16
    tr.struct.count = 3
    k, prio = tr.targets(0.95)
    assert list(k) == [2, 1, 16]
    assert abs(prio[0] - np.log2(101) / 24) < 1e-6 and prio[1] == 0.0


def test_gather_probe_rejects_bad_arguments_before_any_device_call():
    """Every argument check of seraph_gather_probe runs on the host first, so
    it answers SERAPH_EINVAL without a GPU."""
    import ctypes
    lib = C.lib()
    sec = ctypes.c_double(0.0)
    bad = [
        (0, 8, 0, 1.0, 1),            # no values
        (1 << 32, 8, 0, 1.0, 1),      # 2^32 values
        (16, 0, 0, 1.0, 1),           # no gathers
        (16, 12, 0, 1.0, 1),          # not a multiple of 8
        (16, 8, 17, 1.0, 1),          # hot range beyond the values
        (16, 8, 4, 1.5, 1),           # fraction above 1
        (16, 8, 4, -0.1, 1),          # fraction below 0
        (16, 8, 4, 0.5, 0),           # no timed launch
    ]
    for nv, ng, hot, frac, reps in bad:
        rc = lib.seraph_gather_probe(nv, ng, hot, frac, reps, None, ctypes.byref(sec))
        assert rc == C.SERAPH_EINVAL, (nv, ng, hot, frac, reps)
        assert lib.seraph_last_error()
    assert lib.seraph_gather_probe(16, 8, 4, 0.5, 1, None, None) == C.SERAPH_EINVAL


def test_from_csr_rejects_bad_host_offsets_before_any_device_call():
    """Host CSR offsets that do not start at 0 or that decrease are rejected
    with SERAPH_EINVAL before the library touches a device (so without a GPU
    too), each with a message naming the problem."""
    import numpy as np
    col = np.array([1, 2, 0], dtype=np.uint32)
    cases = [
        (np.array([1, 2, 3, 3], dtype=np.uint64), b"row_off[0]"),       # does not start at 0
        (np.array([0, 2, 1, 3], dtype=np.uint64), b"non-decreasing"),   # decreases at v = 1
        (np.array([0, 1, 2, 1], dtype=np.uint64), b"non-decreasing"),   # decreases at the end
    ]
    for ro, what in cases:
        with pytest.raises(C.SeraphError) as ei:
            seraph.Graph.from_csr(3, ro, col)
        assert ei.value.code == C.SERAPH_EINVAL
        assert what in C.lib().seraph_last_error()
    with pytest.raises(C.SeraphError) as ei:
        seraph.Graph.from_csr(0, np.zeros(1, dtype=np.uint64), col)
    assert ei.value.code == C.SERAPH_EINVAL


def test_pinned_fault_injection_hook_arms_and_disarms_without_gpu():
    assert seraph.debug_pinned_bytes() == 0
    seraph.debug_fail_pinned_alloc(3)
    seraph.debug_fail_pinned_alloc(0)
    assert seraph.debug_pinned_bytes() == 0
