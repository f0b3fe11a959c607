"""CPU checks of the C ABI: the library loads, exports every function that
include/labs.h declares, and rejects bad arguments before touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(labs_\w+)\s*\(", text, flags=re.M):
            if "typedef" not in m.group(0) and "#define" not in m.group(0):
                names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2210_15962_gb300 import build
    build.build()
    import paper_2210_15962_gb300 as m
    return m.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["labs_energy", "labs_walks", "labs_saw_round", "labs_walks_workspace_size",
                     "labs_energy_batch", "labs_opts_init", "labs_status_str"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(lib):
    import paper_2210_15962_gb300 as m
    assert m.status_str(m.LABS_OK) == "ok"
    assert m.status_str(m.LABS_EINVAL) == "invalid argument"
    assert m.status_str(12345) == "unknown status"


def test_opts_layout_matches_header(lib):
    import paper_2210_15962_gb300 as m
    o = m.labs_opts()
    lib.labs_opts_init(ctypes.byref(o))
    assert o.target_E == -1 and o.max_rounds == 0 and o.recheck_every == 0 and o.device_buffers == 0


def test_struct_layouts_match_c_compiler(tmp_path):
    # compile a probe against the header with the host C compiler and compare with the ctypes mirrors
    import subprocess
    import paper_2210_15962_gb300 as m
    src = tmp_path / "probe.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "labs.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu\\n", sizeof(labs_opts), sizeof(labs_stats),'
                   ' offsetof(labs_opts, workspace), offsetof(labs_opts, rounds_per_seed),'
                   ' offsetof(labs_stats, device_ms));'
                   'printf("%zu %zu %zu %zu\\n", sizeof(labs_problem), offsetof(labs_problem, target_E),'
                   ' sizeof(labs_batch_opts), offsetof(labs_batch_opts, rounds_per_launch));'
                   'printf("%zu %zu %zu %zu %zu\\n", sizeof(labs_serve_cfg), sizeof(labs_result),'
                   ' offsetof(labs_result, t_done_ns), sizeof(labs_serve_stats), offsetof(labs_serve_stats, status));'
                   'printf("%zu\\n", offsetof(labs_result, p_optimal));'
                   'return 0;}\n')
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [ctypes.sizeof(m.labs_opts), ctypes.sizeof(m.labs_stats), m.labs_opts.workspace.offset,
            m.labs_opts.rounds_per_seed.offset, m.labs_stats.device_ms.offset,
            ctypes.sizeof(m.labs_problem), m.labs_problem.target_E.offset, ctypes.sizeof(m.labs_batch_opts),
            m.labs_batch_opts.rounds_per_launch.offset, ctypes.sizeof(m.labs_serve_cfg),
            ctypes.sizeof(m.labs_result), m.labs_result.t_done_ns.offset, ctypes.sizeof(m.labs_serve_stats),
            m.labs_serve_stats.status.offset, m.labs_result.p_optimal.offset]
    assert got == want


@pytest.mark.parametrize("L", [4, 6, 3, 1, 513, 1001, -7])
def test_walks_rejects_bad_L(lib, L):
    import paper_2210_15962_gb300 as m
    seeds = np.array([1], dtype=np.uint64)
    seq = np.zeros(max(L, 1), dtype=np.int8)
    E = np.zeros(1, dtype=np.int64)
    st = lib.labs_walks(L, m._ptr(seeds), 1, 4, 8, 100, m._ptr(seq), m._ptr(E), None, None)
    assert st == m.LABS_EINVAL
    assert lib.labs_walks_workspace_size(L, 1, 4, 8) == 0


def test_walks_rejects_bad_sizes(lib):
    import paper_2210_15962_gb300 as m
    seeds = np.array([1], dtype=np.uint64)
    seq = np.zeros(27, dtype=np.int8)
    E = np.zeros(1, dtype=np.int64)
    p = m._ptr
    assert lib.labs_walks(27, p(seeds), 0, 4, 8, 100, p(seq), p(E), None, None) == m.LABS_EINVAL  # no seeds
    assert lib.labs_walks(27, p(seeds), 1, 0, 8, 100, p(seq), p(E), None, None) == m.LABS_EINVAL  # no walks
    assert lib.labs_walks(27, p(seeds), 1, 4, 0, 100, p(seq), p(E), None, None) == m.LABS_EINVAL  # no steps
    assert lib.labs_walks(27, p(seeds), 1, 4, 8, 0, p(seq), p(E), None, None) == m.LABS_EINVAL  # no budget
    assert lib.labs_walks(27, None, 1, 4, 8, 100, p(seq), p(E), None, None) == m.LABS_EINVAL  # null seeds
    assert lib.labs_walks(27, p(seeds), 1, 4, 8, 100, None, p(E), None, None) == m.LABS_EINVAL
    assert lib.labs_walks(27, p(seeds), 65536, 65536, 8, 100, p(seq), p(E), None, None) == m.LABS_EINVAL
    o = m.labs_opts()
    lib.labs_opts_init(ctypes.byref(o))
    o.recheck_every = -1
    assert lib.labs_walks(27, p(seeds), 1, 4, 8, 100, p(seq), p(E), ctypes.byref(o), None) == m.LABS_EINVAL
    for bad_kernel in (-1, 5):
        lib.labs_opts_init(ctypes.byref(o))
        o.kernel = bad_kernel
        assert lib.labs_walks(27, p(seeds), 1, 4, 8, 100, p(seq), p(E), ctypes.byref(o), None) == m.LABS_EINVAL


def test_size_arithmetic_does_not_wrap(lib):
    # sizes whose byte counts exceed 64 bits are refused, never wrapped to a
    # small number (argument checks only: no CUDA call is reached)
    import paper_2210_15962_gb300 as m
    big_walks, big_len = (1 << 31) - 1, 1 << 26
    assert lib.labs_walks_workspace_size(511, 1, big_walks, big_len) == 2 ** 64 - 1
    assert lib.labs_walks_workspace_size(121, 1, 4, big_len + 1) == 0    # labs_walks rejects it
    assert lib.labs_walks_workspace_size(121, 65536, 65536, 8) == 0      # more than 2^31 walks
    assert lib.labs_walks_workspace_size(121, 1, 4, 8) > 0
    fake = ctypes.c_void_p(16)  # never dereferenced: the call returns before touching its buffers
    assert lib.labs_saw_round_noalloc(511, 1, 0, big_walks, big_len, fake, fake, None, None, None) == m.LABS_ENOMEM
    assert lib.labs_saw_round_noalloc(27, 1, 0, 4, big_len + 1, fake, fake, None, None, None) == m.LABS_EINVAL
    t = np.zeros(64, dtype=np.int32)
    assert lib.labs_saw_round(27, 1, 0, 4, 8, 0, None, None, None, None, None, m._ptr(t), (1 << 31) - 1, 2, -1,
                              None, 0, None, 0) == m.LABS_EINVAL
    with pytest.raises(m.LabsError) as ei:
        m.Server(max_walk_len=(1 << 26) + 1)
    assert ei.value.status == m.LABS_EINVAL


def test_device_entry_points_refuse_host_tensors(lib):
    # the device-buffer bindings check their tensors before the library sees a pointer
    import torch
    import paper_2210_15962_gb300 as m
    sd = torch.tensor([1], dtype=torch.int64)
    with pytest.raises(m.LabsError) as ei:
        m.labs_walks_device(27, sd, 4, 8, 100, torch.zeros((1, 27), dtype=torch.int8), torch.zeros(1, dtype=torch.int64))
    assert ei.value.status == m.LABS_EINVAL
    with pytest.raises(m.LabsError) as ei:
        m.labs_saw_round_noalloc(27, 1, 0, 4, 8, torch.zeros(4, dtype=torch.int64), torch.zeros(4 * 27, dtype=torch.int8))
    assert ei.value.status == m.LABS_EINVAL
    with pytest.raises(m.LabsError) as ei:
        m.make_opts(workspace=torch.zeros(64, dtype=torch.uint8))
    assert ei.value.status == m.LABS_EINVAL


def test_energy_rejects_bad_args(lib):
    import paper_2210_15962_gb300 as m
    assert lib.labs_energy(None, 5) == m.LABS_EINVAL
    s = np.ones(3, dtype=np.int8)
    assert lib.labs_energy(m._ptr(s), 0) == m.LABS_EINVAL
    assert lib.labs_energy_batch(None, 1, 5, None, None, 1) == m.LABS_EINVAL


def test_saw_round_rejects_bad_args(lib):
    import paper_2210_15962_gb300 as m
    assert lib.labs_saw_round(28, 1, 0, 4, 8, 0, None, None, None, None, None, None, 0, 0, -1, None, 0,
                              None, 0) == m.LABS_EINVAL
    t = np.zeros(64, dtype=np.int32)
    assert lib.labs_saw_round(27, 1, 0, 4, 8, 0, None, None, None, None, None, m._ptr(t), 2, 4, -1, None, 0,
                              None, 0) == m.LABS_EINVAL
    assert lib.labs_saw_round(27, 1, 0, 4, 8, 0, None, None, None, None, None, None, 0, 0, -1, None, 0,
                              None, 5) == m.LABS_EINVAL


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    import paper_2210_15962_gb300 as m
    monkeypatch.setattr(m, "_lib", None)
    monkeypatch.setattr(m, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError, match="not built"):
        m.load()


def test_hex_helpers_roundtrip_table1(lib):
    # the C ABI's Table 1 helpers (host code, no GPU): every printed code decodes
    # to a sequence with the printed energy and encodes back to the same digits
    import paper_2210_15962_gb300 as m
    import oracle
    rows = [l.split() for l in open(os.path.join(ROOT, "tests", "golden", "table1_skew_sequences.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 17
    for r in rows:
        L, E, hx = int(r[0]), int(r[1]), r[4]
        s = m.from_hex(hx, L)
        assert oracle.energy(s) == E
        assert oracle.energy(oracle.skew_expand(s[:(L + 1) // 2], L)) == E and np.array_equal(
            oracle.skew_expand(s[:(L + 1) // 2], L), s)
        assert m.to_hex(s) == hx  # ceil(D/4) digits with the leading zeros Table 1 prints
        assert np.array_equal(m.from_hex("0x" + hx.lower(), L), s)


def test_hex_helpers_reject_bad_input(lib):
    import paper_2210_15962_gb300 as m
    L = 27  # D = 14: at most 0x3FFF
    import oracle
    assert np.array_equal(m.from_hex("0", L), oracle.skew_expand(np.ones(14, dtype=np.int8), L))
    assert m.to_hex(m.from_hex("3FFF", L)) == "3FFF"
    for bad in ["", "0x", "4000", "12G4", "0x-1"]:
        with pytest.raises(m.LabsError) as ei:
            m.from_hex(bad, L)
        assert ei.value.status == m.LABS_EINVAL
    with pytest.raises(m.LabsError):
        m.from_hex("1", 26)  # even L
    s = m.from_hex("2A5", L)
    t = s.copy()
    t[-1] = -t[-1]  # breaks Eq. 2
    with pytest.raises(m.LabsError):
        m.to_hex(t)
    t = s.copy()
    t[0] = 0  # not +-1
    with pytest.raises(m.LabsError):
        m.to_hex(t)
    buf = ctypes.create_string_buffer(4)  # needs ceil(14/4) + 1 = 5 bytes
    assert lib.labs_to_hex(m._ptr(s), L, buf, 4) == m.LABS_EINVAL
    assert lib.labs_to_hex(m._ptr(s), L, buf, 0) == m.LABS_EINVAL
    assert lib.labs_from_hex(None, L, m._ptr(s)) == m.LABS_EINVAL


@pytest.mark.parametrize("bad", [(6, 32, 10, 1, 100), (27, 0, 10, 1, 100), (27, 32, 0, 1, 100), (27, 32, 10, 1, 0),
                                 (513, 32, 10, 1, 100)])
def test_batch_rejects_bad_problems(lib, bad):
    import paper_2210_15962_gb300 as m
    with pytest.raises(m.LabsError) as ei:
        m.Batch([(27, 64, 100, 1, 1000), bad])
    assert ei.value.status == m.LABS_EINVAL


def test_batch_rejects_bad_options(lib):
    import paper_2210_15962_gb300 as m
    for kw in [dict(block_threads=48), dict(block_threads=512), dict(table_factor_x10=5), dict(walk_mode=4)]:
        with pytest.raises(m.LabsError) as ei:
            m.Batch([(27, 64, 100, 1, 1000)], **kw)
        assert ei.value.status == m.LABS_EINVAL


def test_serve_rejects_bad_config(lib):
    import paper_2210_15962_gb300 as m
    for kw in [dict(max_active=0), dict(max_L=100), dict(max_L=1001), dict(rounds_per_launch=0),
               dict(block_threads=40), dict(mem_bytes=0), dict(max_walks=0), dict(walk_mode=3),
               dict(walk_mode=2, max_walks=8192)]:
        with pytest.raises(m.LabsError) as ei:
            m.Server(**kw)
        assert ei.value.status == m.LABS_EINVAL
    assert lib.labs_serve_submit(None, None, None) == m.LABS_EINVAL
    assert lib.labs_serve_poll(None, 1, None, None) == m.LABS_EINVAL
    assert lib.labs_serve_destroy(None) == m.LABS_EINVAL


def test_full_space_rejects_bad_args(lib):
    import paper_2210_15962_gb300 as m
    seeds = np.array([1], dtype=np.uint64)
    seq = np.zeros(300, dtype=np.int8)
    E = np.zeros(1, dtype=np.int64)
    p = m._ptr
    for L in [2, 1, 0, 257, 511]:
        assert lib.labs_walks_full(L, p(seeds), 1, 4, 8, 100, p(seq), p(E), None, None) == m.LABS_EINVAL
        assert lib.labs_walks_full_workspace_size(L, 1, 4, 8) == 0
    o = m.labs_opts()
    lib.labs_opts_init(ctypes.byref(o))
    o.kernel = 2  # the incremental variant is skew-only
    assert lib.labs_walks_full(64, p(seeds), 1, 4, 8, 100, p(seq), p(E), ctypes.byref(o), None) == m.LABS_EINVAL
    assert lib.labs_saw_round_full(257, 1, 0, 4, 8, 0, None, None, None, None, None, None, 0, 0, -1, None, 0,
                                   None) == m.LABS_EINVAL
    # even lengths are fine in the full space and sized like any other
    assert lib.labs_walks_full_workspace_size(64, 1, 4, 8) > 0
    assert lib.labs_walks_workspace_size(64, 1, 4, 8) == 0

