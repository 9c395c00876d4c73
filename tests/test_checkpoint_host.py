"""Checkpoint files of the IMEX-TR outer loop, host side (no GPU): the library's writer and
reader compiled as plain C++ with g++, a bitwise round trip (including a NaN and doubles
that need 17 digits), NumPy and json reading the files, the reader's refusals (a field
of another grid, a truncated field, a missing file, an older format) and the resume check
that refuses a checkpoint written for another problem (box, xi, tau, gamma, precision, eta).
"""
import json
import os
import shutil
import subprocess

import numpy as np
import pytest

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_2603_03933_gb300", "csrc")

HARNESS = r"""
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>
#include "checkpoint.h"
using namespace lbtr;
int main(int argc, char** argv) {
    const std::string path = argv[1];
    const std::string mode = argv[2];
    std::string err;
    if (mode == "write") {
        TrCheckpoint c;
        c.dim = 2; c.n = 8; c.j = 5; c.r = 0.1; c.nu = 1.0 / 3.0; c.mu = 12345.678901234567;
        c.rho_prev = -2.5e-300; c.have_rho = 1; c.random_next = 0; c.rstream = 4000000000u;
        c.accepted = 3; c.contracted = 1; c.shrunk = 1; c.randomized = 2; c.inner = 123456789012LL;
        c.g1_min = std::nan("");
        c.sub_stalled = 2; c.sub_capped = 1; c.sub_worst_rel_res = 3.0e-6;
        c.box[0] = 8.0 * 3.141592653589793; c.box[1] = 0.1 + 0.2; c.xi = 1.0; c.tau = -0.15;
        c.gamma = 0.25; c.eta = 0.1; c.precision = 1;
        std::vector<double> f(64);
        for (int i = 0; i < 64; ++i) f[i] = std::sin(1.0 + i) / 7.0;
        if (!write_checkpoint(path, c, f.data(), 64, err)) { std::printf("ERR %s\n", err.c_str()); return 1; }
        TrCheckpoint d;
        std::vector<double> g;
        if (!read_checkpoint(path, d, g, err)) { std::printf("ERR %s\n", err.c_str()); return 1; }
        bool same = d.dim == 2 && d.n == 8 && d.j == 5 && d.r == c.r && d.nu == c.nu && d.mu == c.mu &&
                    d.rho_prev == c.rho_prev && d.have_rho == 1 && d.random_next == 0 && d.rstream == c.rstream &&
                    d.accepted == 3 && d.contracted == 1 && d.shrunk == 1 && d.randomized == 2 &&
                    d.inner == c.inner && std::isnan(d.g1_min) && g.size() == 64 &&
                    d.sub_stalled == 2 && d.sub_capped == 1 && d.sub_worst_rel_res == c.sub_worst_rel_res &&
                    d.box[0] == c.box[0] && d.box[1] == c.box[1] && d.box[2] == 0.0 && d.xi == 1.0 &&
                    d.tau == c.tau && d.gamma == c.gamma && d.eta == c.eta && d.precision == 1 &&
                    checkpoint_matches(d, c, err) &&
                    std::memcmp(g.data(), f.data(), 64 * sizeof(double)) == 0;
        std::printf(same ? "SAME\n" : "DIFF\n");
        return same ? 0 : 1;
    }
    TrCheckpoint d;
    std::vector<double> g;
    const bool ok = read_checkpoint(path, d, g, err);
    if (ok && mode == "match") {
        // the problem of the written checkpoint, with one value changed (argv[3])
        TrCheckpoint w = d;
        const std::string what = argc > 3 ? argv[3] : "";
        if (what == "box") w.box[1] = std::nextafter(w.box[1], 1.0);
        if (what == "tau") w.tau = -0.1;
        if (what == "gamma") w.gamma = 0.3;
        if (what == "xi") w.xi = 2.0;
        if (what == "precision") w.precision = 0;
        if (what == "eta") w.eta = 0.05;
        if (what == "grid") w.n = 16;
        std::string e2;
        const bool m = checkpoint_matches(d, w, e2);
        std::printf(m ? "MATCH\n" : "MISMATCH %s\n", e2.c_str());
        return 0;
    }
    std::printf(ok ? "READ\n" : "REFUSED %s\n", err.c_str());
    return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("ck")
    src = d / "harness.cpp"
    src.write_text(HARNESS)
    exe = d / "harness"
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", CSRC, "-x", "c++", os.path.join(CSRC, "checkpoint.cu"),
                    "-x", "c++", str(src), "-o", str(exe)], check=True)
    return str(exe)


def test_round_trip_is_bitwise_and_numpy_reads_the_field(harness, tmp_path):
    path = str(tmp_path / "state")
    out = subprocess.run([harness, path, "write"], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "SAME", out.stdout
    field = np.load(path + ".npy")
    assert field.shape == (8, 8) and field.dtype == np.float64
    want = np.sin(1.0 + np.arange(64)) / 7.0
    assert np.max(np.abs(field.ravel() - want)) <= 1e-15
    meta = json.load(open(path + ".json"))
    assert meta["j"] == 5 and meta["nu"] == 1.0 / 3.0 and meta["inner"] == 123456789012
    assert np.isnan(meta["g1_min"])
    assert not os.path.exists(path + ".npy.tmp") and not os.path.exists(path + ".json.tmp")


def test_reader_refuses_other_grids_and_damaged_files(harness, tmp_path):
    path = str(tmp_path / "state")
    subprocess.run([harness, path, "write"], check=True, capture_output=True)
    np.save(path + ".npy", np.zeros((16, 16)))                  # another grid
    out = subprocess.run([harness, path, "read"], capture_output=True, text=True).stdout
    assert out.startswith("REFUSED") and "grid" in out
    np.save(path + ".npy", np.zeros((8, 8)))                    # the right grid reads back
    assert subprocess.run([harness, path, "read"], capture_output=True, text=True).stdout.startswith("READ")
    raw = open(path + ".npy", "rb").read()
    open(path + ".npy", "wb").write(raw[:-8])                   # truncated field
    assert subprocess.run([harness, path, "read"], capture_output=True, text=True).stdout.startswith("REFUSED")
    os.remove(path + ".json")
    assert subprocess.run([harness, path, "read"], capture_output=True, text=True).stdout.startswith("REFUSED")


def test_resume_check_refuses_another_problem(harness, tmp_path):
    path = str(tmp_path / "state")
    subprocess.run([harness, path, "write"], check=True, capture_output=True)
    same = subprocess.run([harness, path, "match", "none"], capture_output=True, text=True).stdout
    assert same.startswith("MATCH"), same
    for what in ("box", "tau", "gamma", "xi", "precision", "eta", "grid"):
        out = subprocess.run([harness, path, "match", what], capture_output=True, text=True).stdout
        assert out.startswith("MISMATCH"), (what, out)
    meta = json.load(open(path + ".json"))
    assert meta["format"] == 2 and meta["precision"] == 1 and meta["tau"] == -0.15
    # a file of the previous format (no problem record) is refused, not resumed blindly
    meta["format"] = 1
    open(path + ".json", "w").write(json.dumps(meta))
    out = subprocess.run([harness, path, "read"], capture_output=True, text=True).stdout
    assert out.startswith("REFUSED") and "format" in out
