"""Host logic of the DRAM-traffic record: parsing of an ncu metrics CSV and the check that a
recorded figure is dropped once the kernel sources change."""
import json

from paper_2604_06309_gb300 import traffic

HEADER = ('"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream","Block Size",'
          '"Grid Size","Device","CC","Section Name","Metric Name","Metric Unit","Metric Value"\n')


def _row(lid, kernel, metric, unit, value):
    return ('"%d","1","python","h","%s","1","7","(512, 1, 1)","(152, 1, 1)","0","10.3","Command line profiler '
            'metrics","%s","%s","%s"\n' % (lid, kernel, metric, unit, value))


def test_parse_takes_the_first_launch_with_both_metrics(tmp_path):
    p = tmp_path / "t.csv"
    p.write_text("program output line\n" + HEADER +
                 _row(0, "k_stage_prep(SolverView, ...)", "dram__bytes_read.sum", "Mbyte", "5.00") +
                 _row(0, "k_stage_prep(SolverView, ...)", "dram__bytes_write.sum", "Mbyte", "1.00") +
                 _row(3, "void k_hi_f64<4, false>(SolverView, ...)", "dram__bytes_read.sum", "Mbyte", "708.94") +
                 _row(3, "void k_hi_f64<4, false>(SolverView, ...)", "dram__bytes_write.sum", "Kbyte",
                      "3,044.61") +
                 _row(9, "void k_hi_f64<4, false>(SolverView, ...)", "dram__bytes_read.sum", "Gbyte", "9.0") +
                 _row(9, "void k_hi_f64<4, false>(SolverView, ...)", "dram__bytes_write.sum", "byte", "1"))
    name, b = traffic.parse_ncu_csv(str(p))
    assert "k_hi_f64" in name
    assert b == 708940000 + 3044610


def test_lookup_drops_a_figure_of_other_kernel_sources(tmp_path, monkeypatch):
    store = tmp_path / "traffic_k_hi.json"
    monkeypatch.setattr(traffic, "STORE", str(store))
    store.write_text(json.dumps({"fp64": {"kernel": "k", "dram_bytes_per_launch": 123, "workload": "w",
                                          "kernel_source_sha16": traffic.source_sha16()},
                                 "df": {"kernel": "k", "dram_bytes_per_launch": 456, "workload": "w",
                                        "kernel_source_sha16": "0" * 16}}))
    assert traffic.lookup("fp64") == 123
    assert traffic.lookup("df") is None
    assert traffic.lookup("fp32") is None
