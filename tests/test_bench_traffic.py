"""bench.py --write-traffic on CPU: ncu --csv launch logs (the column layout
ncu writes) to DRAM bytes per even site per stencil kernel variant, named as
the bench names its kernels, with the commands and the source hash."""
import csv
import json


HDR = ["ID", "Process ID", "Process Name", "Host Name", "Kernel Name", "Context", "Stream", "Block Size",
       "Grid Size", "Device", "CC", "Section Name", "Metric Name", "Metric Unit", "Metric Value"]


def _log(path, launches):
    """launches: (id, kernel name, read bytes, read unit, write bytes, write unit)."""
    with open(path, "w", newline="") as fh:
        fh.write("==PROF== Connected to process 1\n")
        w = csv.writer(fh, quoting=csv.QUOTE_ALL)
        w.writerow(HDR)
        for lid, name, rd, ru, wr, wu in launches:
            base = [str(lid), "1", "python3", "127.0.0.1", name, "1", "7", "(64, 2, 1)", "(24576, 1, 1)", "0",
                    "10.3", "Command line profiler metrics"]
            w.writerow(base + ["dram__bytes_read.sum", ru, rd])
            w.writerow(base + ["dram__bytes_write.sum", wu, wr])
            w.writerow(base + ["gpu__time_duration.sum", "usecond", "361.0"])


def test_traffic_from_ncu_logs(tmp_path):
    import bench
    vh = 32 ** 4 // 2
    f16 = tmp_path / "traffic_f16.csv"
    _log(f16, [(0, "void hop_mr_kernel<3, 1, 1, 0, 0, 2, 2>(HopArgs)", str(1800 * vh), "byte", "0", "byte"),
               (2, "void hop_mr_kernel<3, 1, 1, 1, 0, 2, 2>(HopArgs)", str(2000 * vh), "byte", "0", "byte"),
               (3, "void hop_mr_kernel<3, 1, 2, 1, 2, 2, 3>(HopArgs)", "4", "Gbyte", "2.5", "Gbyte")])
    reset = tmp_path / "traffic_reset.csv"
    _log(reset, [(0, "void hop_kernel_capped3<4, 0, 2, 1, 3>(HopArgs)", "1,000", "Mbyte", "500", "Mbyte")])
    kern = bench.traffic_kernels([str(f16), str(reset)])
    # plain and adjoint pass 1 together: their mean
    p1 = kern["dw_hat_pass1_odd/store/f16/nr2/u12"]
    assert p1["launches"] == 2 and abs(p1["dram_bytes_per_site"] - 1900.0) < 1e-9
    cg = kern["dw_hat_pass2_even/cg_update/f16/nr2/u12"]
    assert abs(cg["dram_bytes_per_site"] - 6.5e9 / vh) < 1e-6
    # double-float kernels read the split binary64 links: link format u64, one rhs per thread
    df = kern["dw_hat_pass2_even/fp64_residual/df64/nr1/u64"]
    assert abs(df["dram_bytes_per_site"] - 1.5e9 / vh) < 1e-6 and df["capture"] == "traffic_reset.csv"
    out = tmp_path / "traffic.json"
    assert bench.write_traffic([str(f16), str(reset)], str(out)) == 0
    d = json.load(open(out))
    assert d["kernels"] == json.loads(json.dumps(kern))
    assert d["source_sha256"] == bench.stencil_source_hash()
    assert d["commands"] == bench.TRAFFIC_COMMANDS and any("--write-traffic" in c for c in d["commands"])
    assert all("--clock-control none" in c for c in d["commands"] if c.startswith("ncu"))


def test_source_hash_ignores_comments_not_code():
    import bench
    src = {f: "int a = 1; // one\n/* block\n comment */ float b;\n" for f in bench.STENCIL_SOURCES}
    h0 = bench.stencil_source_hash(lambda f: src[f])
    commented = dict(src, **{bench.STENCIL_SOURCES[0]: "// header\nint a = 1;   // other words\nfloat b;\n"})
    assert bench.stencil_source_hash(lambda f: commented[f]) == h0
    changed = dict(src, **{bench.STENCIL_SOURCES[0]: "int a = 2; float b;\n"})
    assert bench.stencil_source_hash(lambda f: changed[f]) != h0
    assert bench.traffic_for("dw_hat_pass1_odd/store/f16/nr2/u12") is not None   # the committed capture is current
