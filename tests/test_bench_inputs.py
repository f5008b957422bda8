"""The benchmark's input construction and bookkeeping (CPU): the conserved
variables of the split surface match the oracle's thermodynamics, the
workloads have the stated shapes and ranges, and the algorithmic flop count
per Newton iteration is the stated formula's."""
import numpy as np
import pytest

import bench
import oracle
from paper_2510_10005_gb300 import inputs


@pytest.mark.parametrize("n_p", [4, 7, 15])
def test_flow_state_energy_matches_oracle_thermo(n_p):
    """u = sum Y_i u_i(T) of the split surface's input, for NASA-7 (n_p = 4)
    and for refitted c_p polynomials of other degrees."""
    m = inputs.gen_mechanism("ch4")
    if n_p != 4:
        m = inputs.with_thermo_degree(m, n_p)
    r = oracle.RefMech(m)
    T, Y, p = inputs.field_flames(m, 64, seed=2)
    rho, u, rhoY = bench.flow_state(m, T, Y, p)
    uo = np.array([Y[c] @ r.thermo(T[c])["u"] for c in range(len(T))])
    np.testing.assert_allclose(u, uo, rtol=1e-12, atol=1e-9 * np.abs(uo).max())
    np.testing.assert_allclose(rho, p / (inputs.R_UNIV * T * (Y / m.W).sum(axis=1)), rtol=1e-15)
    np.testing.assert_allclose(rhoY.sum(axis=1), rho * Y.sum(axis=1), rtol=1e-14)


@pytest.mark.parametrize("config,ns,lo,hi", [(1, 9, 1000, 1500), (4, 53, 1100, 1400), (5, 160, 700, 1600)])
def test_workload_ranges(config, ns, lo, hi):
    (m, T, Y, p), = bench.make_workload(config, 256)
    assert m.ns == ns and len(T) == 256 and Y.shape == (256, ns)
    assert T.min() >= lo and T.max() <= hi
    np.testing.assert_allclose(Y.sum(axis=1), 1.0, rtol=1e-12)


def test_flops_per_newton_formula():
    m = inputs.gen_mechanism("ch4")
    n = m.ns + 1
    j = bench.j_term_count(m)
    assert bench.algorithmic_flops_per_newton(m.ns, m.nr, j, False) == \
        pytest.approx(2 * n**3 / 3 + 8 * n * n + 2 * j + 30 * m.nr + 40 * m.ns)
    assert bench.algorithmic_flops_per_newton(m.ns, m.nr, j, True) == \
        pytest.approx(8 * n * n + 2 * j + 30 * m.nr + 40 * m.ns)
    assert 150_000 < bench.algorithmic_flops_per_newton(m.ns, m.nr, j, False) < 160_000



def test_reference_arm_takes_the_workload_options(capsys, monkeypatch):
    """--surface split and --sri-plog change the reference arm's workload
    (the oracle's split step on an SRI/PLOG mechanism) and its stated
    workload, exactly as they change the GPU arm's."""
    import argparse
    import json
    monkeypatch.setenv("WORLD_SIZE", "1")
    monkeypatch.setenv("RANK", "0")
    args = argparse.Namespace(config=1, cells=64, method=None, linear=None, prec=None, surface="split",
                              sri_plog=True, thermo_degree=None, cpu_sample=8, steps=1, warmup=0, gpus=1)
    bench.run_reference(args)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["config"]["workload"] == bench.full_workload_name(args)
    assert "operator-split" in line["config"]["workload"] and "PLOG" in line["config"]["workload"]
    assert line["value"] > 0


def test_adjoint_arms_name_their_workload(capsys, monkeypatch):
    """The adjoint arms (config 4, and config 5 with --adjoint) time the
    oracle's forward + adjoint on the workload they name; the 160-species
    form states its cell count and parameter count."""
    import argparse
    import json
    monkeypatch.setenv("WORLD_SIZE", "1")
    monkeypatch.setenv("RANK", "0")
    args = argparse.Namespace(config=4, cells=64, cpu_sample=2, steps=1, warmup=0, gpus=1, adjoint=False)
    bench.run_reference_adjoint(args)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["metric"] == bench.METRIC_ADJ and line["config"] == {"workload": bench.CONFIGS[4]["workload"],
                                                                      "config": 4}
    assert line["value"] > 0
    w5 = bench.adjoint_workload(5, bench.ADJOINT_CELLS[5])
    assert w5.startswith(bench.CONFIGS[5]["workload"]) and "8,192 cells" in w5 and "2700 Arrhenius" in w5
    m = inputs.gen_mechanism("c7")
    assert 3 * m.nr == 2700


def test_traffic_only_for_the_captured_kernel_sources(monkeypatch):
    """The DRAM traffic of the bench line is the ncu capture's bytes per cell
    scaled to the launch, and null for any workload or kernel source it was
    not taken on."""
    import hashlib
    import os
    h = hashlib.sha256()
    for f in bench.TRAFFIC_SOURCES:
        with open(os.path.join(bench.ROOT, "paper_2510_10005_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    per = bench.TRAFFIC[2]["bytes_per_cell"]
    # at least the 440 B of state read per cell; the writes add the L2
    # scratch slots written back as L2 evicts them (about 13 KB per cell)
    assert 440 < per < 20000
    monkeypatch.setitem(bench.TRAFFIC, 2, dict(bench.TRAFFIC[2], sha256=h.hexdigest()))
    assert bench.measured_traffic(2, 1 << 20) == pytest.approx(per * (1 << 20))
    assert bench.measured_traffic(3, 1 << 20) is None
    monkeypatch.setitem(bench.TRAFFIC, 2, dict(bench.TRAFFIC[2], sha256="0" * 64))
    assert bench.measured_traffic(2, 1 << 20) is None


def test_cpu_baseline_is_a_fixed_sample_and_a_median():
    """cpu_baseline and the reference arm time the same fixed sample of each
    workload (cells evenly spaced through the field) and report the median
    of repeated timings."""
    calls, seq = [], iter([3.0, 1.0, 2.0, 9.0, 2.5])

    def run(k):                       # a stand-in oracle with varying timings
        calls.append(k)
        return next(seq), k
    k, med, times = bench.median_timing(run, 4096, 5)
    assert calls == [4096] * 5 and k == 4096 and med == 2.5 and len(times) == 5
    assert bench.CPU_SAMPLE[2] == 4096 and bench.CPU_SAMPLE[5] == 256 and bench.CPU_SAMPLE[4] == 256
    idx = bench.sample_indices(1 << 20, 4096)
    assert len(idx) == 4096 and idx[0] == 0 and idx[-1] == (1 << 20) - 1 and np.all(np.diff(idx) > 0)
    assert len(bench.sample_indices(100, 4096)) == 100          # never more than every cell
    parts = bench.make_workload(1, 4096)
    v, el, k = bench.cpu_oracle_sample(parts, bench.opts_dict(1, 0), 256, 4)
    assert k == 256 and el > 0 and v == pytest.approx(k / el)
