"""The host walk and layout under AddressSanitizer and UBSan (CPU only).

plan.cpp (with trace.cpp, its phase timer) and a small shim
(tests/sanitize/plan_shim.cpp) are compiled with
-fsanitize=address,undefined and driven, in a child process with the ASan
runtime preloaded, over the test trees, random schemas, forests and the
planning errors (NULL with a count, aliases, cycles).  Any memory error or
undefined behaviour aborts the child.  The shim also checks the relocation
tables the way the relocation kernel reads them (every slot inside its tile,
each record in the group it names, each group's base plus the record's offset
equal to the plan's offset of the target block, and the record's slot being
the one that points at that block).  For span staging it checks the spans and
the placement table on every tree, and on trees from one bump buffer emulates
the whole staged path (span copies, NULL-slot fix-ups, placement) against the
blocks' own bytes."""
import os
import shutil
import subprocess
import sys
import textwrap

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1906_01128_b300", "csrc")
CUDA = "/usr/local/cuda"

DRIVER = textwrap.dedent(r'''
    import ctypes, os, random, sys
    sys.path.insert(0, ROOT)
    import treegen as tg
    from paper_1906_01128_b300 import schema_struct
    lib = ctypes.CDLL(SO)
    lib.shim_plan.restype = ctypes.c_int
    lib.shim_plan.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p]
    lib.shim_message.restype = ctypes.c_char_p

    def plan(schema, roots, pack=0):
        cs, keep = schema_struct(schema)
        arr = (ctypes.c_void_p * len(roots))(*roots)
        out = (ctypes.c_uint64 * 6)()
        rc = lib.shim_plan(ctypes.byref(cs), arr, len(roots), pack, out)
        if rc == 1000:
            raise SystemExit("table check: " + lib.shim_message().decode())
        return rc, list(out)

    trees = [tg.workload("tiny"), tg.node_tree(3, 16, tg.lognormal(300, 1.2, 5000), seed=2),
             tg.node_tree(4, 3, tg.uniform(0, 9), seed=4), tg.linear_tree(6, 100, "llinit", seed=5),
             tg.dense_tree(3, 7, 3, seed=6), tg.listing1_tree(50, seed=7), tg.node_tree(5, 16, 3, seed=1)]
    rng = random.Random(11)
    for i in range(80):
        s, levels, rules = tg.random_schema(rng)
        trees.append(tg.Tree(s, levels, rules, seed=2000 + i))
    n = 0
    for t in trees:
        for pack in (0, 1):  # 16-byte blocks, and small arrays packed at their element alignment
            rc, out = plan(t.schema, [t.root], pack)
            assert rc == 0, (t.name, pack, rc)
        n += out[0]
    forest = tg.batched(40, seed=9, t_max=256 << 10)
    for pack in (0, 1):
        rc, out = plan(forest[0].schema, [t.root for t in forest], pack)
        assert rc == 0, rc
    # targets 64 GiB and more past their lane group's base (reserved address space, never read)
    far = tg.ReservedChain(7, 2 ** 31 - 2)
    rc, out = plan(far.schema, [far.root])
    assert rc == 0 and out[2] == 3 and out[4] == 224 + 7 * 8 * (2 ** 31 - 2), (rc, out)
    # planning errors: the same tree twice in a forest (alias), a NULL root in a forest
    rc, _ = plan(forest[0].schema, [forest[0].root, forest[0].root])
    assert rc != 0
    # span staging: the spans and the placement table of every tree above (their blocks are
    # malloc'd, so nothing reads between them), then the whole staged path emulated on trees
    # whose blocks come from one bump buffer (gaps of 0 to 2,000 bytes: one span or many)
    lib.shim_spans.restype = ctypes.c_int
    lib.shim_spans.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int,
                               ctypes.c_void_p]

    def spans(schema, roots, flags, emulate):
        cs, keep = schema_struct(schema)
        arr = (ctypes.c_void_p * len(roots))(*roots)
        out = (ctypes.c_uint64 * 4)()
        rc = lib.shim_spans(ctypes.byref(cs), arr, len(roots), flags, emulate, out)
        if rc == 1000:
            raise SystemExit("span check: " + lib.shim_message().decode())
        return rc, list(out)

    SPANS, PACK = 16, 8
    for t in trees:
        for fl in (SPANS, SPANS | PACK):
            rc, out = spans(t.schema, [t.root], fl, 0)
            assert rc == 0 and out[0] == 1, (t.name, fl, rc, out)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from bump import BumpAllocator
    keep_alive = []
    rng = random.Random(12)
    for i in range(30):
        s, levels, rules = tg.random_schema(rng)
        sized = tg.Tree(s, levels, rules, seed=2100 + i)  # for the buffer's size
        gap = rng.choice([0, 8, 48, 2000])
        nb = sized.payload_bytes + (1 << 20)
        sized.free()
        b = BumpAllocator(nb + 40000 * (gap + 32), gap)
        t = tg.Tree(s, levels, rules, seed=2100 + i, alloc=b.alloc)
        keep_alive.append(b)
        for fl in (SPANS, SPANS | PACK):
            rc, out = spans(t.schema, [t.root], fl, 1)
            assert rc == 0 and out[0] == 1, (i, fl, rc, out)
    for al in (8,):  # blocks off 16-byte boundaries: the staging keeps each span's phase
        b = BumpAllocator(32 << 20, gap=4, min_align=al)
        keep_alive.append(b)
        t = tg.node_tree(3, 6, tg.uniform(1, 3000), seed=77, alloc=b.alloc)
        assert any(a % 16 for a, _ in b.blocks)
        for fl in (SPANS, SPANS | PACK):
            rc, out = spans(t.schema, [t.root], fl, 1)
            assert rc == 0 and out[0] == 1, (al, fl, rc, out)
    b = BumpAllocator(16 << 20)
    t = tg.node_tree(4, 8, 10, seed=300, alloc=b.alloc)  # 1,244 blocks of 40-byte arrays: by the rule
    rc, out = spans(t.schema, [t.root], 0, 1)
    assert rc == 0 and out[0] == 1 and out[2] == 1, out
    rc, out = spans(t.schema, [t.root], PACK, 1)
    assert rc == 0 and out[0] == 1, out
    print("planned", len(trees) + 1, "trees,", n, "blocks; span staging checked")
''')


def test_plan_under_asan_and_ubsan(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    so = str(tmp_path / "libplan_asan.so")
    cmd = [gxx, "-std=c++17", "-O1", "-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
           "-fno-omit-frame-pointer", "-shared", "-fPIC", f"-I{CUDA}/include", f"-I{CSRC}",
           os.path.join(CSRC, "plan.cpp"), os.path.join(CSRC, "trace.cpp"), os.path.join(CSRC, "spans.cpp"),
           os.path.join(CSRC, "arena.cpp"), os.path.join(CSRC, "debug.cpp"),
           os.path.join(HERE, "sanitize", "plan_shim.cpp"),
           f"-L{CUDA}/lib64", "-lcudart", f"-Wl,-rpath,{CUDA}/lib64", "-o", so]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    asan = subprocess.run([gxx, "-print-file-name=libasan.so"], capture_output=True, text=True).stdout.strip()
    ubsan = subprocess.run([gxx, "-print-file-name=libubsan.so"], capture_output=True, text=True).stdout.strip()
    env = dict(os.environ, LD_PRELOAD=f"{asan}:{ubsan}", ASAN_OPTIONS="detect_leaks=0",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")
    code = f"ROOT = {ROOT!r}\nSO = {so!r}\n" + DRIVER
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, (r.stdout[-3000:], r.stderr[-3000:])
    assert "planned" in r.stdout


def test_thread_pool_under_tsan(tmp_path):
    """The host pool with several callers' jobs in flight at once (the server's slots share one
    pool): every item runs exactly once and every call returns after its own items, under
    ThreadSanitizer."""
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    so = str(tmp_path / "libpool_tsan.so")
    cmd = [gxx, "-std=c++17", "-O1", "-g", "-fsanitize=thread", "-shared", "-fPIC", f"-I{CSRC}",
           os.path.join(HERE, "sanitize", "pool_shim.cpp"), "-lpthread", "-o", so]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    tsan = subprocess.run([gxx, "-print-file-name=libtsan.so"], capture_output=True, text=True).stdout.strip()
    code = textwrap.dedent(f"""
        import ctypes, sys
        lib = ctypes.CDLL({so!r})
        lib.pool_stress.restype = ctypes.c_int
        lib.pool_stress.argtypes = [ctypes.c_uint, ctypes.c_uint, ctypes.c_uint, ctypes.c_uint64]
        lib.pool_message.restype = ctypes.c_char_p
        for threads, callers, jobs, seed in ((4, 1, 200, 1), (4, 6, 120, 2), (8, 8, 80, 3), (2, 3, 150, 4)):
            rc = lib.pool_stress(threads, callers, jobs, seed)
            if rc:
                sys.exit("pool: " + lib.pool_message().decode())
        print("pool ok")
    """)
    env = dict(os.environ, LD_PRELOAD=tsan, TSAN_OPTIONS="halt_on_error=1 report_signal_unsafe=0")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "pool ok" in r.stdout, (r.stdout[-3000:], r.stderr[-3000:])
