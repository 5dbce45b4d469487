// ptrom_save / ptrom_load: a trained PTROM model as one binary file, so the
// offline stages (Sec. 5.1) run once and the online model (Sec. 5.2-5.3)
// is reloaded without retraining.
//
// File layout (native little-endian; both supported hosts are):
//   char[8]  "PTROMMDL"
//   u32      0x01020304 (byte-order check), u32 format version (2; 1 is
//            still read: it has no inflow array)
//   i32 x 8  n_s, M, M_r, N_c, max_gn, qr_prec, built, n
//   f64 x 5  dt, delta, tol, and the origin (ox, oy) the model's FP32
//            coordinates are taken relative to (fixed when the model was
//            created, kept across reparametrisations)
//   arrays, each as u64 element count then the elements:
//     f64 phi_s, x0_s, phi_c, x0_c, gamma_c, A;   i32 off, idx
//     f64 u_s (version 2: the superimposed inflow, 0 or 2 n_s elements)
//   built models only:
//     f64 phi, sigma;  i32 sampled, cl_off, cl_mem;  f64 x0
//   u64      FNV-1a hash of every preceding byte
// Loading checks the tag, version, hash and every array length against the
// sizes, then rebuilds the model through ptrom_model_create.
#include <stdio.h>
#include <string.h>

#include <vector>

#include "ptrom_model.h"

namespace ptrom {
namespace {

constexpr char kMagic[8] = {'P', 'T', 'R', 'O', 'M', 'M', 'D', 'L'};
constexpr unsigned kOrder = 0x01020304u, kVersion = 2u;

struct Writer {
    std::vector<unsigned char> buf;
    void bytes(const void *p, size_t n) {
        const unsigned char *c = (const unsigned char *)p;
        buf.insert(buf.end(), c, c + n);
    }
    template <typename T> void val(T v) { bytes(&v, sizeof(T)); }
    template <typename T> void arr(const std::vector<T> &v) {
        val<unsigned long long>(v.size());
        if (!v.empty()) bytes(v.data(), v.size() * sizeof(T));
    }
};

struct Reader {
    const unsigned char *p;
    size_t n, at = 0;
    bool ok = true;
    bool bytes(void *dst, size_t k) {
        if (!ok || k > n - at) return ok = false;
        memcpy(dst, p + at, k);
        at += k;
        return true;
    }
    template <typename T> T val() {
        T v{};
        bytes(&v, sizeof(T));
        return v;
    }
    // an array whose length must equal `expect`
    template <typename T> std::vector<T> arr(size_t expect) {
        const unsigned long long len = val<unsigned long long>();
        std::vector<T> v;
        if (!ok || len != expect || len > (n - at) / sizeof(T)) {
            ok = false;
            return v;
        }
        v.resize(len);
        if (len) bytes(v.data(), len * sizeof(T));
        return v;
    }
};

unsigned long long fnv1a(const unsigned char *p, size_t n) {
    unsigned long long h = 1469598103934665603ull;
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

}  // namespace
}  // namespace ptrom

using namespace ptrom;

extern "C" int ptrom_save(const ptrom_model *m, const char *path) {
    if (!m || !path) return set_error(PTROM_EINVAL, "ptrom_save: NULL argument");
    const DevModel &d = m->d;
    Writer w;
    w.bytes(kMagic, 8);
    w.val<unsigned>(kOrder);
    w.val<unsigned>(kVersion);
    for (int v : {d.ns, d.M, d.Mr, d.Nc, d.max_gn, m->qr_prec, m->built ? 1 : 0, m->n}) w.val<int>(v);
    for (double v : {d.dt, d.delta, d.tol, m->ox, m->oy}) w.val<double>(v);
    w.arr(m->h_phi_s);
    w.arr(m->h_x0_s);
    w.arr(m->h_phi_c);
    w.arr(m->h_x0_c);
    w.arr(m->h_gamma_c);
    w.arr(m->h_A);
    w.arr(m->h_off);
    w.arr(m->h_idx);
    w.arr(m->h_u_s);
    if (m->built) {
        w.arr(m->phi);
        w.arr(m->sigma);
        w.arr(m->sampled);
        w.arr(m->cl_off);
        w.arr(m->cl_mem);
        w.arr(m->x0_full);
    }
    w.val<unsigned long long>(fnv1a(w.buf.data(), w.buf.size()));
    FILE *f = fopen(path, "wb");
    if (!f) return set_error(PTROM_EINVAL, "ptrom_save: cannot open '%s' for writing", path);
    const size_t put = fwrite(w.buf.data(), 1, w.buf.size(), f);
    const int closed = fclose(f);
    if (put != w.buf.size() || closed != 0) return set_error(PTROM_EINVAL, "ptrom_save: short write to '%s'", path);
    return PTROM_OK;
}

extern "C" int ptrom_load(const char *path, ptrom_model **out) {
    if (!path || !out) return set_error(PTROM_EINVAL, "ptrom_load: NULL argument");
    *out = nullptr;
    FILE *f = fopen(path, "rb");
    if (!f) return set_error(PTROM_EINVAL, "ptrom_load: cannot open '%s'", path);
    std::vector<unsigned char> buf;
    unsigned char chunk[1 << 16];
    size_t got;
    while ((got = fread(chunk, 1, sizeof(chunk), f)) > 0) buf.insert(buf.end(), chunk, chunk + got);
    fclose(f);
    if (buf.size() < 8 + 8 + 8) return set_error(PTROM_EINVAL, "ptrom_load: '%s' is too short", path);
    unsigned long long stored = 0;
    memcpy(&stored, buf.data() + buf.size() - 8, 8);
    if (stored != fnv1a(buf.data(), buf.size() - 8))
        return set_error(PTROM_EINVAL, "ptrom_load: '%s' fails its checksum", path);
    Reader r{buf.data(), buf.size() - 8};
    char magic[8];
    r.bytes(magic, 8);
    if (!r.ok || memcmp(magic, kMagic, 8) != 0) return set_error(PTROM_EINVAL, "ptrom_load: '%s' is not a model", path);
    if (r.val<unsigned>() != kOrder) return set_error(PTROM_EINVAL, "ptrom_load: byte order differs");
    const unsigned ver = r.val<unsigned>();
    if (ver != kVersion && ver != 1u)
        return set_error(PTROM_EINVAL, "ptrom_load: format version %u, expected 1 or %u", ver, kVersion);
    const int ns = r.val<int>(), M = r.val<int>(), Mr = r.val<int>(), Nc = r.val<int>();
    const int max_gn = r.val<int>(), qr_prec = r.val<int>(), built = r.val<int>(), n = r.val<int>();
    const double dt = r.val<double>(), delta = r.val<double>(), tol = r.val<double>();
    const double ox = r.val<double>(), oy = r.val<double>();
    if (!r.ok || ns < 1 || M < 1 || Mr < 1 || Nc < 1 || ns > kMaxNs || M > kMaxM || Mr > kMaxMr || Nc > kMaxNc ||
        (built && (n < ns || n > (1 << 26))))
        return set_error(PTROM_EINVAL, "ptrom_load: bad sizes in header");
    const auto phi_s = r.arr<double>((size_t)2 * ns * M), x0_s = r.arr<double>(2 * (size_t)ns);
    const auto phi_c = r.arr<double>((size_t)2 * Nc * M), x0_c = r.arr<double>(2 * (size_t)Nc);
    const auto gamma_c = r.arr<double>(Nc), A = r.arr<double>((size_t)Mr * 2 * ns);
    const auto off = r.arr<int>(ns + 1);
    const size_t L = (r.ok && off.size() == (size_t)ns + 1 && off[ns] >= 0) ? (size_t)off[ns] : 0;
    const auto idx = r.arr<int>(L);
    std::vector<double> u_s;
    if (ver >= 2u) {  // the inflow array: empty or one value per sampled dof
        const size_t at = r.at;
        const unsigned long long len = r.val<unsigned long long>();
        r.at = at;
        u_s = r.arr<double>(len == 0 ? 0 : 2 * (size_t)ns);
    }
    if (!r.ok) return set_error(PTROM_EINVAL, "ptrom_load: truncated or inconsistent arrays");
    std::vector<double> phi, sigma, x0;
    std::vector<int> sampled, cl_off, cl_mem;
    if (built) {
        phi = r.arr<double>((size_t)2 * n * M);
        sigma = r.arr<double>(M);
        sampled = r.arr<int>(ns);
        cl_off = r.arr<int>(Nc + 1);
        const size_t Lm = (r.ok && cl_off.size() == (size_t)Nc + 1 && cl_off[Nc] >= 0) ? (size_t)cl_off[Nc] : 0;
        cl_mem = r.arr<int>(Lm);
        x0 = r.arr<double>(2 * (size_t)n);
        if (!r.ok) return set_error(PTROM_EINVAL, "ptrom_load: truncated or inconsistent built-model arrays");
        if (cl_off[0] != 0) return set_error(PTROM_EINVAL, "ptrom_load: cluster offsets must start at 0");
        for (int c = 0; c < Nc; ++c)
            if (cl_off[c + 1] < cl_off[c]) return set_error(PTROM_EINVAL, "ptrom_load: cluster offsets not monotone");
        for (int v : cl_mem)
            if (v < 0 || v >= n) return set_error(PTROM_EINVAL, "ptrom_load: cluster member out of range");
        for (int v : sampled)
            if (v < 0 || v >= n) return set_error(PTROM_EINVAL, "ptrom_load: sampled body out of range");
    }
    if (r.at != r.n) return set_error(PTROM_EINVAL, "ptrom_load: trailing bytes in '%s'", path);
    ptrom_model_desc desc{};
    desc.n_s = ns;
    desc.M = M;
    desc.M_r = Mr;
    desc.N_c = Nc;
    desc.dt = dt;
    desc.delta = delta;
    desc.tol = tol;
    desc.max_gn = max_gn;
    desc.qr_prec = qr_prec;
    desc.phi_s = phi_s.data();
    desc.x0_s = x0_s.data();
    desc.phi_c = phi_c.data();
    desc.x0_c = x0_c.data();
    desc.gamma_c = gamma_c.data();
    desc.A = A.data();
    desc.off = off.data();
    desc.idx = idx.empty() ? off.data() : idx.data();
    desc.u_s = u_s.empty() ? nullptr : u_s.data();
    ptrom_model *m = nullptr;
    PTROM_TRY(ptrom_model_create(&desc, &m));
    if (m->ox != ox || m->oy != oy) {  // the saved origin, then the FP32 arrays again
        m->ox = ox;
        m->oy = oy;
        const int e = model_fill_param(m, x0_s.data(), phi_c.data(), x0_c.data(), gamma_c.data());
        if (e != PTROM_OK) {
            ptrom_free(m);
            return e;
        }
    }
    if (built) {
        m->built = true;
        m->n = n;
        m->phi = phi;
        m->sigma = sigma;
        m->sampled = sampled;
        m->A = A;
        m->cl_off = cl_off;
        m->cl_mem = cl_mem;
        const int e = model_store_basis(m, phi.data(), x0.data());
        if (e != PTROM_OK) {
            ptrom_free(m);
            return set_error(e, "ptrom_load: could not store the basis");
        }
    }
    *out = m;
    return PTROM_OK;
}
