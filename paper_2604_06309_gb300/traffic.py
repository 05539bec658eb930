"""DRAM traffic of the history-integral kernels, recorded from ncu captures.

``record`` reads the CSV that ``ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum
... --csv --log-file FILE`` writes (one captured launch of a ``k_hi`` kernel), and stores
read + write bytes of the first captured launch in profiles/traffic_k_hi.json under the
precision's key, with a hash of the kernel sources. ``lookup`` returns the stored bytes
only while that hash still matches the sources, so a figure taken before a kernel change
is never reported for the changed kernel.

    python -m paper_2604_06309_gb300.traffic PRECISION CSV "workload description"
"""
import csv
import hashlib
import json
import os
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
STORE = os.path.join(ROOT, "profiles", "traffic_k_hi.json")
KERNEL_SOURCES = ["kernels_hi.cu", "kernels_df.cu", "hi_units.h", "dmfe_internal.h", "df64.h"]
UNITS = {"byte": 1.0, "kbyte": 1e3, "mbyte": 1e6, "gbyte": 1e9, "tbyte": 1e12}


def source_sha16():
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(PKG, "csrc", name), "rb") as f:
            h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()[:16]


def parse_ncu_csv(path, kernel_prefix="k_hi"):
    """(kernel name, DRAM read + write bytes) of the first captured launch whose name
    contains kernel_prefix."""
    with open(path, newline="") as f:
        lines = [ln for ln in f if ln.startswith('"')]  # skip the program's own output
    rows = list(csv.DictReader(lines))
    launches = {}
    for r in rows:
        name = r.get("Kernel Name", "")
        if kernel_prefix not in name:
            continue
        metric = r.get("Metric Name", "")
        if metric not in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            continue
        unit = UNITS.get(r.get("Metric Unit", "byte").strip().lower())
        if unit is None:
            raise ValueError("unknown unit %r" % r.get("Metric Unit"))
        val = float(r["Metric Value"].replace(",", "")) * unit
        lid = int(r["ID"])
        ent = launches.setdefault(lid, {"name": name, "bytes": 0.0, "n": 0})
        ent["bytes"] += val
        ent["n"] += 1
    full = [k for k in sorted(launches) if launches[k]["n"] == 2]
    if not full:
        raise ValueError("no launch with both DRAM metrics in %s" % path)
    first = launches[full[0]]
    return first["name"], int(round(first["bytes"]))


def record(precision, csv_path, workload):
    name, b = parse_ncu_csv(csv_path)
    store = {}
    if os.path.exists(STORE):
        with open(STORE) as f:
            store = json.load(f)
    store[precision] = {"kernel": name, "dram_bytes_per_launch": b, "workload": workload,
                        "kernel_source_sha16": source_sha16()}
    with open(STORE, "w") as f:
        json.dump(store, f, indent=1, sort_keys=True)
        f.write("\n")
    return store[precision]


def lookup(precision):
    """Stored DRAM bytes per launch for this precision, or None if absent or stale."""
    try:
        with open(STORE) as f:
            ent = json.load(f)[precision]
    except (OSError, KeyError, ValueError):
        return None
    if ent.get("kernel_source_sha16") != source_sha16():
        return None
    return int(ent["dram_bytes_per_launch"])


if __name__ == "__main__":
    print(json.dumps(record(sys.argv[1], sys.argv[2], sys.argv[3])))
