// Checkpoint of the symbolic analysis (Sec. 4.2: the symbolic phase runs once
// per sparsity pattern): the whole Plan written to / read from a file, so a
// later process skips the ordering and the symbolic factorisation.  Format:
// an 8-byte magic and a version, then every field of the Plan in a fixed
// order (scalars as 8-byte values, vectors as an 8-byte element count, the
// element size and the raw little-endian elements), then the magic again.
// Any mismatch on reading is an error; nothing is trusted beyond sizes that
// fit the file.
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "ipm_plan.h"

namespace ipm {

namespace {

constexpr char kMagic[8] = {'I', 'P', 'M', 'P', 'L', 'A', 'N', '1'};
constexpr uint64_t kVersion = 3;

struct Writer {
    FILE *f;
    bool ok = true;
    void raw(const void *p, size_t n) {
        if (ok && n && std::fwrite(p, 1, n, f) != n) ok = false;
    }
    template <class T>
    void scalar(T &v) {
        static_assert(std::is_arithmetic<T>::value, "scalar");
        int64_t u = 0;
        double d = 0.0;
        if (std::is_floating_point<T>::value) {
            d = (double)v;
            raw(&d, 8);
        } else {
            u = (int64_t)v;
            raw(&u, 8);
        }
    }
    template <class T>
    void vec(std::vector<T> &v) {
        uint64_t n = v.size(), es = sizeof(T);
        raw(&n, 8);
        raw(&es, 8);
        raw(v.data(), n * sizeof(T));
    }
};

struct Reader {
    FILE *f;
    uint64_t left;  // bytes remaining in the file
    bool ok = true;
    void raw(void *p, size_t n) {
        if (!ok) return;
        if (n > left || (n && std::fread(p, 1, n, f) != n)) {
            ok = false;
            return;
        }
        left -= n;
    }
    template <class T>
    void scalar(T &v) {
        if (std::is_floating_point<T>::value) {
            double d = 0.0;
            raw(&d, 8);
            v = (T)d;
        } else {
            int64_t u = 0;
            raw(&u, 8);
            v = (T)u;
        }
    }
    template <class T>
    void vec(std::vector<T> &v) {
        uint64_t n = 0, es = 0;
        raw(&n, 8);
        raw(&es, 8);
        if (!ok || es != sizeof(T) || n > left / sizeof(T)) {
            ok = false;
            return;
        }
        v.resize(n);
        raw(v.data(), n * sizeof(T));
    }
};

// Every field of the Plan, in one order for both directions.
template <class IO>
void visit(Plan &P, IO &io) {
    io.scalar(P.m), io.scalar(P.n), io.scalar(P.N), io.scalar(P.form), io.scalar(P.ordering);
    io.vec(P.Acp), io.vec(P.Ari);
    io.scalar(P.batch_count), io.vec(P.inst);
    io.vec(P.perm), io.vec(P.iperm), io.vec(P.parent), io.vec(P.colcount);
    io.scalar(P.nsuper), io.vec(P.sn_start), io.vec(P.sn_parent), io.vec(P.sn_rptr), io.vec(P.sn_rows);
    io.vec(P.sn_k), io.vec(P.sn_f), io.vec(P.sn_ld), io.vec(P.sn_level), io.vec(P.sn_off);
    io.scalar(P.front_doubles), io.vec(P.child_ptr), io.vec(P.child_list), io.vec(P.map_off), io.vec(P.relmap);
    io.vec(P.orig_ptr), io.vec(P.orig_dst), io.vec(P.orig_src), io.vec(P.sign);
    io.scalar(P.nlevels), io.vec(P.lvl_small_ptr), io.vec(P.lvl_small), io.vec(P.lvl_large_ptr), io.vec(P.lvl_large);
    io.vec(P.sn_large);
    io.vec(P.upd_off), io.scalar(P.upd_total);
    io.scalar(P.nnzL), io.scalar(P.nnzK_lower), io.scalar(P.flops), io.scalar(P.amalg_zero_frac);
    io.scalar(P.max_f), io.scalar(P.max_k), io.scalar(P.nsmall), io.scalar(P.nlarge);
    io.vec(P.ne_cp), io.vec(P.ne_ri), io.vec(P.ne_tptr), io.vec(P.ne_ta), io.vec(P.ne_tb), io.vec(P.ne_tj);
    io.scalar(P.est_as), io.scalar(P.est_ne), io.scalar(P.nnz_ne_seen);
}

// The read plan must be self-consistent where the device code relies on it.
bool consistent(const Plan &P) {
    const size_t ns = (size_t)P.nsuper;
    if (P.N != P.m + P.n && !(P.form == 2 && P.N == P.m)) return false;
    if (P.perm.size() != (size_t)P.N || P.iperm.size() != (size_t)P.N || P.sign.size() != (size_t)P.N) return false;
    if (P.sn_start.size() != ns + 1 || P.sn_rptr.size() != ns + 1 || P.sn_k.size() != ns || P.sn_f.size() != ns ||
        P.sn_ld.size() != ns || P.sn_off.size() != ns + 1 || P.sn_parent.size() != ns ||
        P.child_ptr.size() != ns + 1 || P.map_off.size() != ns + 1 || P.orig_ptr.size() != ns + 1 ||
        P.upd_off.size() != ns + 1 || P.sn_large.size() != ns)
        return false;
    if (P.sn_rows.size() != (size_t)P.sn_rptr[ns] || P.orig_dst.size() != (size_t)P.orig_ptr[ns] ||
        P.orig_src.size() != P.orig_dst.size() || P.Acp.size() != (size_t)P.n + 1 ||
        P.Ari.size() != (size_t)P.Acp[P.n])
        return false;
    for (size_t s = 0; s < ns; s++) {
        if (P.sn_k[s] < 1 || P.sn_f[s] < P.sn_k[s] || P.sn_ld[s] < P.sn_f[s] ||
            P.sn_rptr[s + 1] - P.sn_rptr[s] != P.sn_f[s] || P.sn_start[s + 1] - P.sn_start[s] != P.sn_k[s] ||
            P.sn_off[s] < 0 || P.sn_off[s] + (int64_t)P.sn_f[s] * P.sn_ld[s] > P.front_doubles)
            return false;
    }
    for (int32_t r : P.sn_rows)
        if (r < 0 || r >= P.N) return false;
    return true;
}

}  // namespace

int plan_save(const Plan &Pc, const std::string &path, std::string &err) {
    FILE *f = std::fopen(path.c_str(), "wb");
    if (!f) {
        err = "cannot open " + path;
        return -1;
    }
    Plan &P = const_cast<Plan &>(Pc);  // visit() is shared with reading; writing does not modify
    Writer w{f};
    uint64_t ver = kVersion;
    w.raw(kMagic, 8);
    w.raw(&ver, 8);
    visit(P, w);
    w.raw(kMagic, 8);
    const bool ok = w.ok && std::fclose(f) == 0;
    if (!ok) err = "write failed: " + path;
    return ok ? 0 : -1;
}

int plan_load(Plan &P, const std::string &path, std::string &err) {
    FILE *f = std::fopen(path.c_str(), "rb");
    if (!f) {
        err = "cannot open " + path;
        return -1;
    }
    std::fseek(f, 0, SEEK_END);
    const long size = std::ftell(f);
    std::fseek(f, 0, SEEK_SET);
    Reader r{f, size > 0 ? (uint64_t)size : 0};
    char magic[8] = {};
    uint64_t ver = 0;
    r.raw(magic, 8);
    r.raw(&ver, 8);
    Plan Q;
    if (r.ok && std::memcmp(magic, kMagic, 8) == 0 && ver == kVersion) visit(Q, r);
    else r.ok = false;
    char tail[8] = {};
    r.raw(tail, 8);
    std::fclose(f);
    if (!r.ok || std::memcmp(tail, kMagic, 8) != 0 || r.left != 0 || !consistent(Q)) {
        err = "not a valid analysis file: " + path;
        return -1;
    }
    P = std::move(Q);
    return 0;
}

}  // namespace ipm
