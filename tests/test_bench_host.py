"""Host logic of bench.py (CPU): the byte models and the stored-traffic lookup."""
import json
import os

import numpy as np

import bench


def test_byte_models():
    n, s = (1024, 1024), 4
    N = n[0] * n[1]
    spec = 6 * (n[0] // 2 + 1) * n[1] * 2 * s
    mb = bench.model_bytes(2, n, s, 1)
    assert mb["pass_a"] == 5 * 6 * N * s + N * s + spec
    assert mb["pass_c"] == 2 * spec and mb["pass_e"] == spec + 2 * 6 * N * s
    mb3 = bench.model_bytes(3, (64, 64, 64), 8, 1)
    assert set(mb3) == {"pass_a", "pass_b", "pass_c", "pass_d", "pass_e"}
    nod = bench.model_bytes(3, (64, 64, 64), 4, 1, "nodal")
    assert nod["force_stencil"] == (6 * 3 + 1) * 64 ** 3 * 4
    # the nodal form moves far fewer bytes than the stress form
    assert sum(nod.values()) < 0.2 * sum(bench.model_bytes(3, (64, 64, 64), 4, 1).values())


def test_traffic_rows_follow_the_kernel_hash(tmp_path):
    h = bench.kernel_source_hash()
    assert len(h) == 16 and all(c in "0123456789abcdef" for c in h)
    rows = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))["entries"]
    assert rows
    for e in rows:
        kind, dim = e["kernel"].rsplit("_", 1)
        got = bench.measured_traffic(e["workload"], e["form"], kind, int(dim[0]))
        if e["source_hash"] == h:
            assert np.isclose(got, e["bytes_per_launch"])
        else:
            assert got is None
    assert bench.measured_traffic("gauss1024", "stress", "no_such_pass", 2) is None
    # an entry counts only under the hash it was taken with
    p = tmp_path / "t.json"
    ent = {"workload": "w", "form": "stress", "kernel": "pass_a_3d", "bytes_per_launch": 5.0}
    p.write_text(json.dumps({"entries": [dict(ent, source_hash=h)]}))
    assert bench.measured_traffic("w", "stress", "pass_a", 3, path=str(p)) == 5.0
    p.write_text(json.dumps({"entries": [dict(ent, source_hash="0" * 16)]}))
    assert bench.measured_traffic("w", "stress", "pass_a", 3, path=str(p)) is None


def test_source_hash_ignores_comments():
    src = 'int a = 1; // note\n/* block\n comment */ const char* s = "x // y /* z */";\nchar q = \'"\';\n\n  \nint b;'
    assert bench.strip_comments(src) == 'int a = 1;\n const char* s = "x // y /* z */";\nchar q = \'"\';\nint b;'
    assert bench.strip_comments("a; // one\na;") == bench.strip_comments("a;\na; // two")
    assert bench.strip_comments("a = 1;") != bench.strip_comments("a = 2;")


def test_scope_model_bytes():
    # 256^3, FP32 fields and spectra: (8 * 4 + 8 * 4) * 36 * N + 4 N = 38.7 GB per CG iteration
    N = 256 ** 3
    assert bench.scope_model_bytes(3, (256,) * 3, 4, 4, 4) == (64 * 36 + 4) * N
    assert abs(bench.scope_model_bytes(3, (256,) * 3, 4, 4, 4) / 1e9 - 38.72) < 0.01
    assert bench.scope_model_bytes(2, (1024, 1024), 8, 8, 8) == (8 * 8 + 4 * 8) * 6 * 1024 ** 2 + 8 * 1024 ** 2


def test_oracle_error_uses_the_stored_result():
    d = bench.golden("disc32")
    C = np.array(d["C_eff"])
    e = bench.oracle_error("disc32", C=C * (1 + 1e-12))
    assert e["value"] < 2e-12 and "tangent" in e["quantity"]
    assert bench.oracle_error("no_such_workload", C=C) is None


def test_oracle_iterations_at_reads_the_residual_history(monkeypatch):
    stored = {"tol": 1e-12, "iterations": [6, 5],
              "rel_residual_history": [[1.0, 0.3, 2e-8, 5e-10, 1e-11, 1e-12, 9e-13],
                                       [1.0, 1e-9, 1e-10, 1e-11, 1e-12, 5e-13]]}
    monkeypatch.setattr(bench, "golden", lambda name: stored)
    assert bench.oracle_iterations_at("x", 1e-9) == ([3, 1], 1e-9)
    assert bench.oracle_iterations_at("x", 1e-8) == ([3, 1], 1e-8)
    assert bench.oracle_iterations_at("x", 1e-12) == ([5, 4], 1e-12)
    # tighter than the stored solve: its own counts, at its own tolerance
    assert bench.oracle_iterations_at("x", 1e-13) == ([6, 5], 1e-12)
    del stored["rel_residual_history"]
    assert bench.oracle_iterations_at("x", 1e-9) == ([6, 5], 1e-12)
    monkeypatch.setattr(bench, "golden", lambda name: {})
    assert bench.oracle_iterations_at("x", 1e-9) == (None, None)


def test_host_cpu_description():
    h = bench.host_cpu()
    assert isinstance(h["model"], str) and h["model"] and h["nproc"] >= 1
    x86 = "processor\t: 0\nmodel name\t: Some CPU @ 3.0GHz\nflags\t: fpu\n"
    assert bench.host_cpu(x86)["model"] == "Some CPU @ 3.0GHz"
    arm = "processor\t: 0\nBogoMIPS\t: 2000.00\nCPU implementer\t: 0x41\nCPU part\t: 0xd4f\n"
    assert bench.host_cpu(arm)["model"].endswith("CPU part 0xd4f")


def test_hbm_fractions():
    mb = bench.model_bytes(2, (1024, 1024), 4, 1)
    # pass A moving its model bytes for 100 load-case iterations in 10 ms at a 6000 GB/s peak
    kt = {"pass_a": (10.0, 50), "pass_c": (0.0, 0), "residual": (1.0, 3), "pass_e": (5.0, 50)}
    f = bench.hbm_fractions(mb, kt, 100.0, 1, 6000.0)
    assert set(f) == {"pass_a", "pass_e"}               # untimed and non-model kernels left out
    assert np.isclose(f["pass_a"], mb["pass_a"] * 100 / 10e-3 / 1e9 / 6000.0)
    assert np.isclose(f["pass_e"] / f["pass_a"], (mb["pass_e"] / 5.0) / (mb["pass_a"] / 10.0))


def test_extension_workloads_inputs():
    for name in bench.EXTENSIONS:
        x = bench.extension_inputs(name)
        assert x["E"].shape == tuple(reversed(x["n"])) and np.all(x["E"] >= 0) and np.any(x["E"] > 0)
        assert x["prec"] in ("mixed", "fp64")
        # finite strain and the other derivatives run in FP64 only
        if "Fm" in x or "derivative" in x:
            assert x["prec"] == "fp64"
        if "Fm" in x:
            assert x["Fm"].shape == (1, len(x["n"]), len(x["n"]))
        else:
            assert x["Em"].shape == (3 if len(x["n"]) == 2 else 6,) * 2
    assert (bench.extension_inputs("porous1024")["E"] == 0).mean() > 0.2
    assert not set(bench.EXTENSIONS) & set(bench.WORKLOADS)


def test_iteration_bytes_per_form():
    # the stress form uses the scope table's model; the other forms their own per-kernel model
    n = (256, 256, 256)
    b, note = bench.iteration_bytes(3, n, 4, "stress", {})
    assert b == bench.scope_model_bytes(3, n, 4, 4, 4) and "8 vector" in note
    mb = bench.model_bytes(3, n, 4, 1, "nodal")
    b2, note2 = bench.iteration_bytes(3, n, 4, "nodal", mb)
    assert b2 == sum(mb.values()) and "nodal" in note2 and b2 < 0.2 * b
