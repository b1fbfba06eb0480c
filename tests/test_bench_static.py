"""bench.py is only run in full on a GPU; this CPU check catches a name that
is used but never defined (a helper lost in an edit) before that run."""
import ast
import builtins
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_uses_no_undefined_names():
    tree = ast.parse(open(os.path.join(ROOT, "bench.py")).read())
    defined = set(dir(builtins)) | {"__file__"}
    for node in ast.walk(tree):
        if isinstance(node, (ast.FunctionDef, ast.ClassDef)):
            defined.add(node.name)
        elif isinstance(node, ast.Import):
            defined.update((a.asname or a.name).split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom):
            defined.update(a.asname or a.name for a in node.names)
        elif isinstance(node, ast.Name) and isinstance(node.ctx, ast.Store):
            defined.add(node.id)
        elif isinstance(node, ast.arg):
            defined.add(node.arg)
        elif isinstance(node, ast.ExceptHandler) and node.name:
            defined.add(node.name)
    used = {n.id for n in ast.walk(tree) if isinstance(n, ast.Name) and isinstance(n.ctx, ast.Load)}
    assert sorted(used - defined) == []


def _bench():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_traffic_line_is_ignored_once_the_kernel_sources_change(tmp_path, monkeypatch):
    """The roofline's DRAM traffic comes from a committed ncu line only while
    the digest of the kernel's sources matches it; it is scaled to the run's
    algorithmic bytes; a stale digest gives None."""
    b = _bench()
    digest = b.kernel_source_digest("k_cg_mtm32_v4a<32,2>")
    assert len(digest) == 12
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "x.md").write_text(
        "traffic_per_launch: k_cg_mtm32_v4a<32,2> %s 1000 2000\n" % digest)
    monkeypatch.setattr(b, "ROOT", str(tmp_path))
    monkeypatch.setattr(b, "kernel_source_digest", lambda k: digest)
    assert b.traffic_from_profiles("k_cg_mtm32_v4a<32,2>", 4000) == 2000.0
    monkeypatch.setattr(b, "kernel_source_digest", lambda k: "0" * 12)
    assert b.traffic_from_profiles("k_cg_mtm32_v4a<32,2>", 4000) is None


def test_every_profiled_kernel_has_a_source_digest():
    """Each kernel named on a committed traffic line is found in csrc/
    (including kernels whose launch bounds hold parentheses), so a stale
    line is detected instead of silently matching nothing."""
    import glob
    b = _bench()
    names = set()
    for path in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        for line in open(path):
            if line.startswith("traffic_per_launch:"):
                names.add(line.split()[1])
    assert names
    for k in sorted(names):
        assert b.kernel_source_digest(k) is not None, k
    assert b.kernel_source_digest("k_cg_update<float,0>") is not None


def test_single_rank_job_rate_and_replica_inputs():
    """At N = 1 the job rate is units over the rank's time; each rank draws
    its own seeded inputs (replicas, no shared data)."""
    import holstein_inputs as hi
    b = _bench()
    assert b.job_rate(1, 32, 500.0) == 64.0
    w = hi.Workload("r", L=4, Ltau=4, seed=3)
    x0, r0 = b.replica_inputs(w, 2, 0)
    x1, r1 = b.replica_inputs(w, 2, 1)
    xa, ra = b.replica_inputs(w, 2, 0)
    assert (x0 == xa).all() and (r0 == ra).all()
    assert not (x0 == x1).all() and not (r0 == r1).all()


def test_bench_line_is_strict_json():
    """Non-finite numbers (a failed trajectory's dH) become null, so the
    printed line parses as strict JSON."""
    import json
    b = _bench()
    obj = {"a": float("inf"), "b": [1.5, float("nan"), {"c": -float("inf")}], "d": 2, "e": "x"}
    out = b.strict_json(obj)
    assert out == {"a": None, "b": [1.5, None, {"c": None}], "d": 2, "e": "x"}
    json.loads(json.dumps(out, allow_nan=False))


def test_profile_summaries_name_their_commands_and_committed_files_only():
    """Every committed ncu summary gives the command that made it, clock
    control off, and runs committed files only (no scratch scripts)."""
    import glob
    files = sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md")))
    assert files
    for path in files:
        text = open(path).read()
        assert "Command" in text, path
        assert "_work" not in text, path
        joined = text.replace("\\\n", " ")   # shell line continuations
        for line in joined.splitlines():
            if line.strip().startswith("ncu "):
                assert "--clock-control none" in line, (path, line)
