"""Host-side logic of bench.py that needs no GPU: the key of the stored construction traffic.

The ncu traffic figure is valid for the kernel code it was captured on.  bench.py keys it to a
hash of the construction kernel's sources without comments and blank lines: an edit of comments
keeps the key, an edit of code changes it (and the bench then reports null traffic)."""
import importlib.util
import os
import shutil

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_code_hash_ignores_comments_and_blank_lines_only(tmp_path):
    b = _bench()
    csrc = tmp_path / "paper_1709_03187_gb300" / "csrc"
    csrc.mkdir(parents=True)
    names = b.CONSTRUCT_SOURCES
    for name in names:
        shutil.copy(os.path.join(ROOT, "paper_1709_03187_gb300", "csrc", name), csrc / name)
    b.ROOT = str(tmp_path)
    h0 = b.code_sha1(*names)
    for name in names:
        text = (csrc / name).read_text()
        (csrc / name).write_text("// a new header comment\n\n" + text.replace("\n", "  // note\n", 3))
        assert b.code_sha1(*names) == h0, name
        (csrc / name).write_text(text)
    # a code edit in either file changes the key
    dev = (csrc / names[0]).read_text()
    (csrc / names[0]).write_text(dev.replace("#define FULL 0xffffffffu", "#define FULL 0xfffffffeu"))
    assert b.code_sha1(*names) != h0
    (csrc / names[0]).write_text(dev)
    host = (csrc / names[1]).read_text()
    (csrc / names[1]).write_text(host.replace("A.n = p.n;", "A.n = p.n + 0;"))
    assert b.code_sha1(*names) != h0


def test_construct_byte_model():
    """Per decision 3 x 4k + 4 B, per exhausted step 8m + 4M B, per rebuilt city 8 + 32 B."""
    b = _bench()
    assert b.construct_bytes_model(1, 0, 0, 16, 1024) == 12 * 16 + 4 + 40
    assert b.construct_bytes_model(0, 1, 1000, 16, 1024) == 8 * 1024 + 4 * 1000
    # the 200,000-city line: about 1e6 decisions, 6e4 exhausted steps with M about 1,000
    assert 0.9e9 < b.construct_bytes_model(10 ** 6, 6 * 10 ** 4, 6 * 10 ** 7, 16, 1024) < 1.1e9
    assert b.construct_bytes_layout(1, 16, 0) == 8 * 16 + 4 + 40


def test_every_name_read_is_bound_somewhere():
    """A coarse lint of the scripts that only run on a GPU machine: every name the module reads is
    bound somewhere in it (an assignment, argument, import, function or class) or is a builtin, so
    a workload cannot fail on a NameError there."""
    import ast
    import builtins
    import pathlib

    root = pathlib.Path(__file__).resolve().parent.parent
    for rel in ("bench.py", "__graft_entry__.py"):
        tree = ast.parse((root / rel).read_text())
        bound = set(dir(builtins)) | {"__file__", "__name__"}
        for node in ast.walk(tree):
            if isinstance(node, (ast.FunctionDef, ast.AsyncFunctionDef, ast.ClassDef)):
                bound.add(node.name)
            elif isinstance(node, ast.arg):
                bound.add(node.arg)
            elif isinstance(node, (ast.Import, ast.ImportFrom)):
                bound.update((a.asname or a.name).split(".")[0] for a in node.names)
            elif isinstance(node, ast.Name) and isinstance(node.ctx, (ast.Store, ast.Del)):
                bound.add(node.id)
            elif isinstance(node, ast.ExceptHandler) and node.name:
                bound.add(node.name)
        used = {n.id for n in ast.walk(tree) if isinstance(n, ast.Name) and isinstance(n.ctx, ast.Load)}
        assert not used - bound, (rel, sorted(used - bound))


def test_every_cuda_unit_is_built():
    """Every .cu file under csrc is a unit of the library build (a unit left out would leave its
    launches undefined at link time only on the machine that builds it)."""
    import importlib
    import pathlib

    build = importlib.import_module("paper_1709_03187_gb300.build")
    csrc = pathlib.Path(ROOT) / "paper_1709_03187_gb300" / "csrc"
    assert {p.name for p in csrc.glob("*.cu")} == {u for u, _ in build.UNITS}


def test_workload_descriptions_follow_the_generators():
    import aco_synth

    b = _bench()
    assert b.instance_desc(aco_synth.WORKLOADS["lbest200k"]) == "clustered (200 Gaussian clusters, sigma=0.005)"
    assert b.instance_desc(aco_synth.WORKLOADS["lbest10k"]).startswith("half uniform in [0,1)^2, half in 20")
    assert b.instance_desc(aco_synth.WORKLOADS["dense100"]) == "uniform in [0,1)^2"
