// Checkpoint files of the IMEX-TR outer loop: host code only (compiles as plain C++ too).
#include "checkpoint.h"

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>

namespace lbtr {

namespace {

std::string shape_text(int dim, int n) {
    std::string s = "(";
    for (int a = 0; a < dim; ++a) s += std::to_string(n) + ", ";
    if (dim == 1) return s + ")";
    s.resize(s.size() - 2);
    return s + ")";
}

bool write_file(const std::string& path, const std::string& head, const void* data, size_t bytes,
                std::string& err) {
    const std::string tmp = path + ".tmp";
    FILE* f = std::fopen(tmp.c_str(), "wb");
    if (!f) { err = "checkpoint: cannot open " + tmp; return false; }
    bool ok = std::fwrite(head.data(), 1, head.size(), f) == head.size();
    if (ok && bytes) ok = std::fwrite(data, 1, bytes, f) == bytes;
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) { err = "checkpoint: write to " + tmp + " failed"; std::remove(tmp.c_str()); return false; }
    if (std::rename(tmp.c_str(), path.c_str()) != 0) {
        err = "checkpoint: cannot rename " + tmp;
        std::remove(tmp.c_str());
        return false;
    }
    return true;
}

bool read_all(const std::string& path, std::string& out, std::string& err) {
    FILE* f = std::fopen(path.c_str(), "rb");
    if (!f) { err = "checkpoint: cannot open " + path; return false; }
    out.clear();
    char buf[1 << 16];
    size_t k;
    while ((k = std::fread(buf, 1, sizeof(buf), f)) > 0) out.append(buf, k);
    const bool bad = std::ferror(f) != 0;
    std::fclose(f);
    if (bad) { err = "checkpoint: read of " + path + " failed"; return false; }
    return true;
}

// the number after "key": in a flat JSON object written by write_checkpoint
bool json_number(const std::string& js, const char* key, double& v) {
    const std::string k = std::string("\"") + key + "\":";
    const size_t p = js.find(k);
    if (p == std::string::npos) return false;
    const char* s = js.c_str() + p + k.size();
    while (*s == ' ') ++s;
    if (std::strncmp(s, "NaN", 3) == 0) { v = std::numeric_limits<double>::quiet_NaN(); return true; }
    char* end = nullptr;
    v = std::strtod(s, &end);
    return end != s;
}

bool little_endian() {
    const uint16_t one = 1;
    unsigned char b;
    std::memcpy(&b, &one, 1);
    return b == 1;
}

}  // namespace

bool write_checkpoint(const std::string& path, const TrCheckpoint& c, const double* field, long long count,
                      std::string& err) {
    if (!little_endian()) { err = "checkpoint: big-endian hosts are not supported"; return false; }
    // NumPy format 1.0: magic, version, header length (uint16 LE), header padded with spaces
    // to a multiple of 64 bytes overall and ended by a newline
    std::string dict = "{'descr': '<f8', 'fortran_order': False, 'shape': " + shape_text(c.dim, c.n) + ", }";
    const size_t pre = 10;
    size_t total = pre + dict.size() + 1;
    const size_t pad = (64 - total % 64) % 64;
    dict.append(pad, ' ');
    dict.push_back('\n');
    std::string head("\x93NUMPY\x01\x00", 8);
    head.push_back((char)(dict.size() & 0xff));
    head.push_back((char)((dict.size() >> 8) & 0xff));
    head += dict;
    if (!write_file(path + ".npy", head, field, (size_t)count * sizeof(double), err)) return false;
    char js[2048];
    auto num = [](double x) {
        if (std::isnan(x)) return std::string("NaN");
        char b[40];
        std::snprintf(b, sizeof(b), "%.17g", x);
        return std::string(b);
    };
    std::snprintf(js, sizeof(js),
                  "{\"format\": 2, \"dim\": %d, \"n\": %d, \"j\": %d, \"r\": %s, \"nu\": %s, \"mu\": %s, "
                  "\"rho_prev\": %s, \"have_rho\": %d, \"random_next\": %d, \"rstream\": %u, \"accepted\": %d, "
                  "\"contracted\": %d, \"shrunk\": %d, \"randomized\": %d, \"inner\": %lld, \"g1_min\": %s, "
                  "\"sub_stalled\": %d, \"sub_capped\": %d, \"sub_worst_rel_res\": %s, \"box_x\": %s, "
                  "\"box_y\": %s, \"box_z\": %s, \"xi\": %s, \"tau\": %s, \"gamma\": %s, \"eta\": %s, "
                  "\"precision\": %d}\n",
                  c.dim, c.n, c.j, num(c.r).c_str(), num(c.nu).c_str(), num(c.mu).c_str(), num(c.rho_prev).c_str(),
                  c.have_rho, c.random_next, c.rstream, c.accepted, c.contracted, c.shrunk, c.randomized, c.inner,
                  num(c.g1_min).c_str(), c.sub_stalled, c.sub_capped, num(c.sub_worst_rel_res).c_str(),
                  num(c.box[0]).c_str(), num(c.box[1]).c_str(), num(c.box[2]).c_str(), num(c.xi).c_str(),
                  num(c.tau).c_str(), num(c.gamma).c_str(), num(c.eta).c_str(), c.precision);
    return write_file(path + ".json", js, nullptr, 0, err);
}

bool read_checkpoint(const std::string& path, TrCheckpoint& c, std::vector<double>& field, std::string& err) {
    if (!little_endian()) { err = "checkpoint: big-endian hosts are not supported"; return false; }
    std::string js;
    if (!read_all(path + ".json", js, err)) return false;
    constexpr int NK = 28;
    double v[NK];
    const char* keys[NK] = {"format", "dim", "n", "j", "r", "nu", "mu", "rho_prev", "have_rho", "random_next",
                            "rstream", "accepted", "contracted", "shrunk", "randomized", "inner", "g1_min",
                            "sub_stalled", "sub_capped", "sub_worst_rel_res", "box_x", "box_y", "box_z", "xi",
                            "tau", "gamma", "eta", "precision"};
    if (!json_number(js, keys[0], v[0])) { err = "checkpoint: no \"format\" in " + path + ".json"; return false; }
    if (v[0] != 2.0) {
        err = "checkpoint: " + path + ".json has format " + std::to_string((int)v[0]) +
              ", not 2 (an older file does not record the problem it belongs to)";
        return false;
    }
    for (int i = 1; i < NK; ++i)
        if (!json_number(js, keys[i], v[i])) { err = std::string("checkpoint: no \"") + keys[i] + "\" in " + path + ".json"; return false; }
    c.dim = (int)v[1]; c.n = (int)v[2]; c.j = (int)v[3];
    c.r = v[4]; c.nu = v[5]; c.mu = v[6]; c.rho_prev = v[7];
    c.have_rho = (int)v[8]; c.random_next = (int)v[9]; c.rstream = (unsigned)v[10];
    c.accepted = (int)v[11]; c.contracted = (int)v[12]; c.shrunk = (int)v[13]; c.randomized = (int)v[14];
    c.inner = (long long)v[15]; c.g1_min = v[16];
    c.sub_stalled = (int)v[17]; c.sub_capped = (int)v[18]; c.sub_worst_rel_res = v[19];
    c.box[0] = v[20]; c.box[1] = v[21]; c.box[2] = v[22];
    c.xi = v[23]; c.tau = v[24]; c.gamma = v[25]; c.eta = v[26]; c.precision = (int)v[27];
    if (c.dim < 1 || c.dim > 3 || c.n < 1) { err = "checkpoint: bad grid in " + path + ".json"; return false; }
    std::string raw;
    if (!read_all(path + ".npy", raw, err)) return false;
    if (raw.size() < 10 || raw.compare(0, 6, "\x93NUMPY", 6) != 0 || raw[6] != 1) {
        err = "checkpoint: " + path + ".npy is not a NumPy 1.0 file";
        return false;
    }
    const size_t hl = (size_t)(unsigned char)raw[8] | ((size_t)(unsigned char)raw[9] << 8);
    if (raw.size() < 10 + hl) { err = "checkpoint: truncated " + path + ".npy"; return false; }
    const std::string dict = raw.substr(10, hl);
    const std::string want = "'shape': " + shape_text(c.dim, c.n);
    if (dict.find("'descr': '<f8'") == std::string::npos || dict.find("'fortran_order': False") == std::string::npos ||
        dict.find(want) == std::string::npos) {
        err = "checkpoint: " + path + ".npy does not hold the grid of " + path + ".json";
        return false;
    }
    long long count = 1;
    for (int a = 0; a < c.dim; ++a) count *= c.n;
    if (raw.size() - 10 - hl != (size_t)count * sizeof(double)) {
        err = "checkpoint: " + path + ".npy has the wrong size";
        return false;
    }
    field.resize((size_t)count);
    std::memcpy(field.data(), raw.data() + 10 + hl, (size_t)count * sizeof(double));
    return true;
}

bool checkpoint_matches(const TrCheckpoint& c, const TrCheckpoint& want, std::string& err) {
    auto bad = [&](const char* what) {
        err = std::string("checkpoint: written for another ") + what;
        return false;
    };
    if (c.dim != want.dim || c.n != want.n) return bad("grid");
    for (int a = 0; a < want.dim; ++a)
        if (c.box[a] != want.box[a]) return bad("box");
    if (c.xi != want.xi) return bad("xi");
    if (c.tau != want.tau) return bad("tau");
    if (c.gamma != want.gamma) return bad("gamma");
    if (c.precision != want.precision) return bad("precision");
    if (c.eta != want.eta) return bad("subproblem step eta");
    return true;
}

}  // namespace lbtr
