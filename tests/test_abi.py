"""The C-ABI library builds, loads and exports every symbol the header declares;
host-side argument checks answer with error codes (no GPU needed)."""
import ctypes as C
import re
from pathlib import Path

import numpy as np
import pytest

ROOT = Path(__file__).resolve().parent.parent


@pytest.fixture(scope="module")
def L():
    from paper_2108_02997_gb300 import binding
    return binding.lib()


def declared_functions():
    names = []
    for h in sorted((ROOT / "include").glob("*.h")):
        text = h.read_text()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*\b(pr_[a-z0-9_]+)\s*\(", text, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for need in ("pr_graph_create", "pr_graph_destroy", "pr_solve", "pr_solve_batch", "pr_last_error"):
        assert need in names


def test_every_declared_symbol_is_exported(L):
    from paper_2108_02997_gb300 import binding
    for name in declared_functions():
        assert hasattr(L, name), f"{name} declared in include/ but not exported"
        assert name in binding.SIGNATURES, f"{name} has no binding signature"


def test_version_and_status_strings(L):
    assert L.pr_version() >= 10000
    assert L.pr_status_string(1) == b"PR_EINVAL"


def _create(L, n, off, src, od):
    h = C.c_void_p()
    off = np.ascontiguousarray(off, np.int32)
    src = np.ascontiguousarray(src, np.int32)
    od = np.ascontiguousarray(od, np.int32)
    st = L.pr_graph_create(n, src.size, off.ctypes.data, src.ctypes.data if src.size else None,
                           od.ctypes.data, C.byref(h))
    return st, h


def test_malformed_csr_is_rejected_before_any_device_work(L):
    """The O(n) checks run on the host before anything touches a device; the
    per-edge checks (source range, per-vertex counts) run on the device and are
    covered by the GPU tests."""
    # non-monotone offsets
    st, _ = _create(L, 3, [0, 2, 1, 3], [1, 2, 0], [1, 1, 1])
    assert st == 1 and b"non-decreasing" in L.pr_last_error()
    # out-degrees that do not add up to the number of edges
    st, _ = _create(L, 2, [0, 1, 1], [1], [0, 0])
    assert st == 1 and b"does not sum" in L.pr_last_error()
    # negative out-degree
    st, _ = _create(L, 2, [0, 1, 1], [1], [2, -1])
    assert st == 1 and b"negative" in L.pr_last_error()
    # offsets[n] != nnz
    st, _ = _create(L, 2, [0, 1, 3], [1], [0, 1])
    assert st == 1
    # offsets[0] != 0
    st, _ = _create(L, 2, [1, 1, 1], [], [0, 0])
    assert st == 1
    # n < 1
    h = C.c_void_p()
    assert L.pr_graph_create(0, 0, None, None, None, C.byref(h)) == 1


def test_solve_rejects_bad_handles_and_arguments(L):
    from paper_2108_02997_gb300 import binding
    out = np.empty(4)
    bogus = C.c_void_p(0x1234)
    assert L.pr_solve(None, 0.85, 1e-6, 1, 500, None, out.ctypes.data, None, None, None) == 5
    assert L.pr_solve(bogus, 0.85, 1e-6, 1, 500, None, out.ctypes.data, None, None, None) == 5
    assert L.pr_graph_destroy(None) == 0
    assert L.pr_graph_destroy(bogus) == 5
    o = binding.default_options()
    o.precision = 17
    assert L.pr_solve_batch(None, 0, C.byref(o)) == 1
    o = binding.default_options()
    o.max_passes = -1
    assert L.pr_solve_batch(None, 0, C.byref(o)) == 1 and b"max_passes" in L.pr_last_error()
    o = binding.default_options()
    o.group = 7
    assert L.pr_solve_batch(None, 0, C.byref(o)) == 1 and b"group" in L.pr_last_error()
    o = binding.default_options()
    o.kernels = 3
    assert L.pr_solve_batch(None, 0, C.byref(o)) == 1 and b"kernels" in L.pr_last_error()
    o = binding.default_options()
    o.loop = 4
    assert L.pr_solve_batch(None, 0, C.byref(o)) == 1 and b"loop" in L.pr_last_error()
    assert L.pr_solve_batch(None, -1, None) == 1


def test_options_defaults(L):
    from paper_2108_02997_gb300 import binding
    o = binding.default_options()
    assert o.precision == binding.PR_PREC_DF64 and o.switch_tol == 1e-6 and o.share_trajectories == 1
    assert o.loop == binding.PR_LOOP_AUTO and o.init == binding.PR_INIT_UNIFORM
    assert o.group == binding.PR_GROUP_AUTO and o.max_passes == 0


def test_learned_start_calls_reject_bad_arguments_before_device_work(L):
    """The warm-start entry points check handles and arguments first (no GPU
    is touched on these paths)."""
    h = C.c_void_p()
    assert L.pr_mlp_create(None, C.byref(h)) == 1
    bad = np.zeros(4609, np.float32)
    bad[17] = np.nan
    assert L.pr_mlp_create(bad.ctypes.data, C.byref(h)) == 1 and b"finite" in L.pr_last_error()
    assert not h.value
    bogus = C.c_void_p(0x1234)
    out = np.empty(8)
    assert L.pr_mlp_warm_start(bogus, bogus, 0.85, out.ctypes.data, None) == 5
    assert L.pr_mlp_warm_start(bogus, bogus, 0.85, None, None) == 1
    assert L.pr_mlp_warm_start(bogus, bogus, 1.5, out.ctypes.data, None) == 1
    feat = np.empty(40, np.float32)
    assert L.pr_features(bogus, 0.85, feat.ctypes.data, None) == 5
    assert L.pr_mlp_loss_grad(bogus, bogus, 0.85, out.ctypes.data, None, None, None) == 5
    assert L.pr_mlp_train(bogus, None, None, None, 1, 1, C.c_float(1e-3), None, None) == 5
    assert L.pr_mlp_destroy(None) == 0
    assert L.pr_mlp_destroy(bogus) == 5


def _struct_fields(text, name):
    """(type, field) pairs of a `typedef struct name { ... } name;` in a header."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    m = re.search(r"typedef struct " + name + r" \{(.*?)\} " + name + ";", text, flags=re.S)
    assert m, name
    out = []
    for decl in m.group(1).split(";"):
        decl = " ".join(decl.split())
        if not decl:
            continue
        f = re.match(r"(.*?)\**\s*\b([a-z_0-9]+)(\[\d+\])?$", decl)
        assert f, decl
        out.append(f.group(2))
    return out


def test_options_and_instance_layouts_match_the_header():
    """The binding's pr_options and pr_instance mirror the header's structures
    field by field and byte by byte (both compilers lay them out the same)."""
    from paper_2108_02997_gb300 import binding as Bd
    text = (ROOT / "include" / "pagerank.h").read_text()
    for name, cls in (("pr_options", Bd.pr_options), ("pr_instance", Bd.pr_instance)):
        assert _struct_fields(text, name) == [f[0] for f in cls._fields_], name
    assert C.sizeof(Bd.pr_instance) == 80 and C.sizeof(Bd.pr_options) % 8 == 0


def test_header_describes_the_workspace_pool_and_its_release():
    """The header's device-memory convention names what the library keeps
    between calls and how to return it (the workspace pool, pr_workspace_info,
    pr_workspace_release), and the no-alloc entry point's limits."""
    text = (ROOT / "include" / "pagerank.h").read_text()
    conv = text[:text.index("#ifndef PAGERANK_H")]
    assert "stream-ordered" in conv and "16 GiB" in conv and "graph pool" in conv
    assert "pr_workspace_info" in conv and "pr_workspace_release" in conv
    assert "cudaMalloc with cudaMalloc" not in conv and "releases it\n *     before returning" not in conv
    noalloc = text[text.index("pr_solve_noalloc —"):text.index("pr_status pr_solve_noalloc(")]
    assert "captured" in noalloc and "40 MiB" in noalloc and "device memory of that device" in noalloc


def test_loop_modes_and_their_options():
    """The binding's loop names map to the header's pr_loop values, the
    persistent wait bound reaches pr_options, and an unknown loop name is
    refused before any library call."""
    from paper_2108_02997_gb300 import binding
    text = (ROOT / "include" / "pagerank.h").read_text()
    for name, value in (("graph", 0), ("host", 1), ("persistent", 2), ("auto", 3)):
        assert binding.LOOPS[name] == value
        assert f"PR_LOOP_{name.upper()} = {value}" in text
        o, _ = binding._make_options(loop=name, persist_wait_us=1234)
        assert o.loop == value and o.persist_wait_us == 1234
    with pytest.raises(ValueError):
        binding._make_options(loop="spin")
    # the header states the bound of the waits and the rule-count limit
    persist = text[text.index("PR_LOOP_PERSISTENT = 2"):text.index("PR_LOOP_AUTO = 3")]
    assert "2 s" in persist and "256 stopping rules" in persist
