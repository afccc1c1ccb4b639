"""The C-ABI library builds, loads without a GPU and exports every declared entry point."""
import os
import re

import pytest

import oracle
from paper_1910_04658_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(bs_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    build.build()
    L = binding.lib()
    decl = declared_functions()
    assert "bs_sketch" in decl and "bs_topk" in decl and "bs_estimate_pairs" in decl
    for name in decl:
        assert hasattr(L, name), name
    assert sorted(n for n, _, _ in binding.SIGNATURES) == decl


def test_host_only_calls():
    build.build()
    assert binding.bs_version() >= 100
    assert binding.bs_status_string(0) == "ok"
    # the library's SplitMix64 seeding agrees with the oracle's own implementation
    for seed in (0, 1, 2**40 + 3, 2**64 - 1):
        assert binding.bs_hash_params(seed) == oracle.hash_params(seed)


def test_env_variant_override_in_plan():
    # bs_topk_plan is host-only: the environment override is visible without a GPU
    import subprocess
    import sys
    code = ("import sys; sys.path.insert(0, '.'); "
            "from paper_1910_04658_gb300 import binding as B; "
            "print(int(B.bs_topk_plan(100000, 100000, 4096, 50, 0, True)[0]))")
    env = dict(__import__("os").environ)
    env.pop("BS_VARIANT", None)
    root = __import__("os").path.dirname(__import__("os").path.dirname(__import__("os").path.abspath(__file__)))
    plain = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, cwd=root)
    env["BS_VARIANT"] = "popc"
    forced = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, cwd=root)
    assert plain.stdout.strip() == "1" and forced.stdout.strip() == "0", (plain.stderr, forced.stderr)


def test_tensor_core_plan_parts_match_the_persistent_schedule():
    # bs_topk_plan is host-only; without a GPU the library assumes 148 SMs.
    # The default tensor-core configuration for N = 4096, k = 50 reads FP4
    # copies of both operands: R = rbs // G rounds of whole 128-row blocks go
    # to the G blocks first (block c: row blocks [c R, (c + 1) R)), the rows
    # left over (fewer row blocks than G) run as a second launch.  When the
    # database's FP4 copy (N / 2 bytes a row) is over 64 MiB, that launch cuts
    # each row block's T 240-row database tiles into P = min(G // rbs, T)
    # equal parts, one block per part, so every row block has P partial lists;
    # otherwise its U = row blocks x T units are dealt out as equal contiguous
    # ranges, block c starting at unit ceil(c U / G): unit x then sits in
    # block floor(x G / U), and the parts of a row block are the blocks it
    # spans.
    from paper_1910_04658_gb300 import binding as B

    G = 148

    def parts(nq, ndb):   # the default configuration's database tiles have 240 rows
        rbs, T = (nq + 127) // 128, (ndb + 239) // 240
        if ndb * 4096 // 2 > 64 << 20:
            return max(1, min(G // rbs, T))
        U = rbs * T
        g = min(G, U)
        first = lambda x: (x * g) // U
        return max(first(rb * T + T - 1) - first(rb * T) + 1 for rb in range(rbs))

    for nq, ndb in ((100_000, 100_000), (4096, 1_000_000), (1000, 1000), (37, 20_000), (129, 257),
                    (148 * 128 * 2, 3000), (148 * 128 * 2 - 5, 3000)):
        for same in (True, False):
            if same and nq != ndb:
                continue
            uses_tc, splits, launches = B.bs_topk_plan(nq, ndb, 4096, 50, B.BS_VARIANT_TC, same)
            rbs = (nq + 127) // 128
            rounds = rbs // G
            q_split = min(nq, rounds * G * 128)
            rest = nq - q_split
            want = parts(rest, ndb) if rest > 0 else 1
            assert uses_tc and splits == want, (nq, ndb, splits, want)
            # the FP4 copies (one for all-pairs), the rounds launch, the
            # launch over the rest, the merge of its partial lists
            assert launches == 1 + (0 if same else 1) + (rounds > 0) + (rest > 0) + (want > 1), (nq, ndb)


def test_batched_plan_claims_whole_row_blocks():
    # bs_topk_batched_plan is host-only (the addresses are never touched): the
    # dynamic schedule never splits a row block, so there is no merge -- one
    # re-layout launch and the ranking launch; an all-empty table launches nothing
    from paper_1910_04658_gb300 import binding as B

    def job(nq, ndb, N, base):
        return dict(Q=base, pcQ=base + 0x100000, DB=base, pcDB=base + 0x100000, score=base + 0x200000,
                    idx=base + 0x300000, nQ=nq, nDB=ndb, N=N, exclude_self=nq == ndb)

    tab = [job(100_000, 100_000, 4096, 1 << 32), job(300, 300, 256, 2 << 32), job(5000, 20, 8192, 3 << 32)]
    assert B.bs_topk_batched_plan(tab, 50) == (1, 2)
    assert B.bs_topk_batched_plan([job(0, 10, 1024, 1 << 32)], 50) == (1, 0)
    # workspace: a 256-byte counter, then per job the larger of its tiled Q
    # (rows to 128) and DB (rows to 208) and its FP4 copies (DB, and Q unless
    # Q is DB: N / 2 bytes a row)
    ws = B.bs_topk_batched_workspace_bytes(tab, 50)
    a256 = lambda x: (x + 255) // 256 * 256

    def per_job(nq, ndb, N):
        tiled = a256(-(-nq // 128) * 128 * N // 8) + a256(-(-ndb // 208) * 208 * N // 8)
        fp4 = a256(ndb * N // 2) + (0 if nq == ndb else a256(nq * N // 2))
        return max(tiled, fp4)
    want = 256 + sum(per_job(nq, ndb, N) for nq, ndb, N in ((100_000, 100_000, 4096), (300, 300, 256), (5000, 20, 8192)))
    assert ws == want, (ws, want)
    with pytest.raises(B.BinSketchError):   # N = 96: not a tensor-core shape
        B.bs_topk_batched_plan([job(10, 10, 96, 1 << 32)], 50)


def test_header_is_plain_c_and_a_c_program_links(tmp_path):
    # the boundary is usable from C: the header compiles as pedantic C99, a
    # program taking the address of every declared function links against the
    # library, and its host-only calls run without a GPU
    import subprocess
    build.build()
    decl = declared_functions()
    src = tmp_path / "caller.c"
    src.write_text(
        '#include <inttypes.h>\n#include <stdio.h>\n#include "binsketch.h"\n'
        "typedef void (*any_fn)(void);\n"
        "static any_fn table[] = {" + ", ".join(f"(any_fn){n}" for n in decl) + "};\n"
        "int main(void) {\n"
        "    uint64_t m = 0, a = 0;\n"
        "    bs_hash_params(12345, &m, &a);\n"
        '    printf("%d %zu %" PRIu64 " %" PRIu64 " %s\\n", bs_version(), sizeof(table) / sizeof(table[0]),\n'
        "           m, a, bs_status_string(BS_ERR_ROWPTR));\n"
        "    return 0;\n}\n")
    lib_dir = os.path.dirname(binding.LIB_PATH)
    exe = tmp_path / "caller"
    r = subprocess.run(["gcc", "-std=c99", "-pedantic", "-Wall", "-Wextra", "-Werror", "-I",
                        os.path.join(ROOT, "include"), str(src), "-L", lib_dir, "-lbinsketch",
                        f"-Wl,-rpath,{lib_dir}", "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stderr
    ver, n, m, a, *status = out.stdout.split()
    assert int(ver) >= 100 and int(n) == len(decl)
    assert (int(m), int(a)) == oracle.hash_params(12345)
    assert " ".join(status) == "malformed row offsets"
