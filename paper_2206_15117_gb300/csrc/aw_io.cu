// Persistence of the library's objects, written by host code with explicit
// little-endian encoding (the same bytes on every host).
//
// aw_surrogate_save / aw_surrogate_load: the surrogate's configuration,
// FP32 parameters, per-w-plane rejection state and engine in one file.
// Layout (every field little-endian, no padding):
//   "AWSURR01"                                  8 bytes
//   int32 npol, width, n_hidden, norm_nw, engine, freq_mode
//   float32 omega0, out_scale
//   float64 D, w_max, f_c, f_h, chi_c, chi_h
//   uint64 seed
//   int32 norm_supports[norm_nw]
//   int64 nparam, float32 params[nparam]
//   int32 nrej, uint8 plane_rejected[nrej]
//   uint64 checksum (FNV-1a 64 of every byte before it)
//
// aw_kernel_set_save / aw_kernel_set_load: a kernel set with its tables in
// their storage format and layout.  Layout:
//   "AWKSET01", the canonical spec encoding (encode_spec), float32 scale,
//   int32 n_rejected, int64 total_elems, int32 elem_bytes,
//   uint64 FNV-1a 64 of every byte before it,
//   the table bytes, uint64 word hash of the table bytes (table_hash).
// aw_kernel_spec_hash is the FNV-1a 64 of the canonical spec encoding of the
// spec after the library's own normalisation (the cache key of a set).
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "aw_internal.h"
#include "aw_mlp.h"

namespace {

const char kMagic[8] = {'A', 'W', 'S', 'U', 'R', 'R', '0', '1'};

struct Writer {
    std::vector<unsigned char> b;
    void raw(const void *p, size_t n) {
        const unsigned char *c = static_cast<const unsigned char *>(p);
        b.insert(b.end(), c, c + n);
    }
    void u64(uint64_t v) {
        for (int i = 0; i < 8; ++i) b.push_back((unsigned char)(v >> (8 * i)));
    }
    void u32(uint32_t v) {
        for (int i = 0; i < 4; ++i) b.push_back((unsigned char)(v >> (8 * i)));
    }
    void i32(int32_t v) { u32((uint32_t)v); }
    void i64(int64_t v) { u64((uint64_t)v); }
    void f32(float v) {
        uint32_t u;
        std::memcpy(&u, &v, 4);
        u32(u);
    }
    void f64(double v) {
        uint64_t u;
        std::memcpy(&u, &v, 8);
        u64(u);
    }
};

struct Reader {
    const std::vector<unsigned char> &b;
    size_t pos = 0;
    bool ok = true;
    explicit Reader(const std::vector<unsigned char> &buf) : b(buf) {}
    bool need(size_t n) {
        if (!ok || b.size() - pos < n) ok = false;
        return ok;
    }
    uint64_t u64() {
        if (!need(8)) return 0;
        uint64_t v = 0;
        for (int i = 0; i < 8; ++i) v |= (uint64_t)b[pos + i] << (8 * i);
        pos += 8;
        return v;
    }
    uint32_t u32() {
        if (!need(4)) return 0;
        uint32_t v = 0;
        for (int i = 0; i < 4; ++i) v |= (uint32_t)b[pos + i] << (8 * i);
        pos += 4;
        return v;
    }
    int32_t i32() { return (int32_t)u32(); }
    int64_t i64() { return (int64_t)u64(); }
    float f32() {
        const uint32_t u = u32();
        float v;
        std::memcpy(&v, &u, 4);
        return v;
    }
    double f64() {
        const uint64_t u = u64();
        double v;
        std::memcpy(&v, &u, 8);
        return v;
    }
};

uint64_t fnv1a(const unsigned char *p, size_t n) {
    uint64_t h = 1469598103934665603ull;
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

}  // namespace

// ---------------------------------------------------------------- kernel sets
namespace {

// Canonical encoding of a normalised spec (arrays inline, in field order).
void encode_spec(const aw_kernel_spec &sp, Writer &w) {
    w.i32(sp.N);
    w.f64(sp.dl);
    w.i32(sp.OS);
    w.f64(sp.W);
    w.i32(sp.npol);
    w.i32(sp.nw);
    w.f64(sp.w_max);
    for (int i = 0; i < sp.nw; ++i) w.i32(sp.supports[i]);
    w.i32(sp.npa);
    for (int i = 0; i < sp.npa; ++i) w.f64(sp.pa[i]);
    w.i32(sp.nfb);
    for (int i = 0; i < sp.nfb; ++i) w.f64(sp.fbin_freqs[i]);
    w.f64(sp.dish_d);
    w.f64(sp.d_xy[0]);
    w.f64(sp.d_xy[1]);
    w.f64(sp.d_yx[0]);
    w.f64(sp.d_yx[1]);
    w.f64(sp.eps);
    w.i32(sp.role);
    w.i32(sp.storage);
    w.f64(sp.point_l);
    w.f64(sp.point_m);
    w.i32(sp.ntype);
    if (sp.ntype >= 2)
        for (int i = 0; i < 4 * sp.ntype; ++i) w.f64(sp.type_leak[i]);
}

// A spec decoded from a file, with its arrays.
struct DecodedSpec {
    aw_kernel_spec sp{};
    std::vector<int32_t> supports;
    std::vector<double> pa, fb, tl;
};

bool decode_spec(Reader &r, DecodedSpec &d) {
    aw_kernel_spec &sp = d.sp;
    sp.N = r.i32();
    sp.dl = r.f64();
    sp.OS = r.i32();
    sp.W = r.f64();
    sp.npol = r.i32();
    sp.nw = r.i32();
    sp.w_max = r.f64();
    if (!r.ok || sp.nw < 1 || sp.nw > 256) return false;
    d.supports.resize(sp.nw);
    for (auto &v : d.supports) v = r.i32();
    sp.npa = r.i32();
    if (!r.ok || sp.npa < 1 || sp.npa > 65535) return false;
    d.pa.resize(sp.npa);
    for (auto &v : d.pa) v = r.f64();
    sp.nfb = r.i32();
    if (!r.ok || sp.nfb < 1 || sp.nfb > 65535) return false;
    d.fb.resize(sp.nfb);
    for (auto &v : d.fb) v = r.f64();
    sp.dish_d = r.f64();
    sp.d_xy[0] = r.f64();
    sp.d_xy[1] = r.f64();
    sp.d_yx[0] = r.f64();
    sp.d_yx[1] = r.f64();
    sp.eps = r.f64();
    sp.role = r.i32();
    sp.storage = r.i32();
    sp.point_l = r.f64();
    sp.point_m = r.f64();
    sp.ntype = r.i32();
    if (!r.ok || sp.ntype < 0 || sp.ntype > 16) return false;
    if (sp.ntype >= 2) {
        d.tl.resize(4 * (size_t)sp.ntype);
        for (auto &v : d.tl) v = r.f64();
    }
    sp.supports = d.supports.data();
    sp.pa = d.pa.data();
    sp.fbin_freqs = d.fb.data();
    sp.type_leak = d.tl.empty() ? nullptr : d.tl.data();
    return r.ok;
}

// Word-wise hash of the table bytes (8 bytes per step, the tail zero-padded).
struct TableHash {
    uint64_t h = 1469598103934665603ull;
    void add(const unsigned char *p, size_t n) {
        size_t i = 0;
        for (; i + 8 <= n; i += 8) {
            uint64_t v;
            std::memcpy(&v, p + i, 8);
            h = (h ^ v) * 1099511628211ull;
            h ^= h >> 29;
        }
        if (i < n) {
            uint64_t v = 0;
            std::memcpy(&v, p + i, n - i);
            h = (h ^ v) * 1099511628211ull;
            h ^= h >> 29;
        }
    }
};

constexpr size_t kIoChunk = (size_t)256 << 20;   // bytes per host staging chunk
const char kSetMagic[8] = {'A', 'W', 'K', 'S', 'E', 'T', '0', '1'};

}  // namespace

int aw_kernel_set_geometry(const aw_kernel_spec *spec, aw_kernel_set *ks);
int aw_kernel_set_alloc(aw_kernel_set *ks);

extern "C" int aw_kernel_spec_hash(const aw_kernel_spec *spec, uint64_t *hash) {
    try {
        if (!spec || !hash) return aw_set_error(AW_EINVAL, "NULL argument");
        aw_kernel_set tmp;
        int rc = aw_kernel_set_geometry(spec, &tmp);
        if (rc) return rc;
        Writer w;
        encode_spec(tmp.spec, w);
        *hash = fnv1a(w.b.data(), w.b.size());
        return AW_OK;
    } catch (const std::bad_alloc &) {
        return aw_set_error(AW_ENOMEM, "host allocation failed");
    } catch (...) {
        return aw_set_error(AW_EINVAL, "unexpected C++ exception");
    }
}

extern "C" int aw_kernel_set_save(const aw_kernel_set *k, const char *path) {
    try {
        if (!k || !path) return aw_set_error(AW_EINVAL, "NULL argument");
        AW_CUDA_TRY(cudaSetDevice(k->device));
        AW_CUDA_TRY(cudaDeviceSynchronize());
        Writer w;
        w.raw(kSetMagic, 8);
        encode_spec(k->spec, w);
        w.f32(k->scale);
        w.i32(k->n_rejected);
        w.i64(k->total_elems);
        w.i32(k->elem_bytes);
        w.u64(fnv1a(w.b.data(), w.b.size()));
        FILE *f = std::fopen(path, "wb");
        if (!f) return aw_set_error(AW_EINVAL, "cannot open '%s' for writing", path);
        bool ok = std::fwrite(w.b.data(), 1, w.b.size(), f) == w.b.size();
        const size_t total = (size_t)k->total_elems * (size_t)k->elem_bytes;
        std::vector<unsigned char> buf(std::min(total, kIoChunk) + 8);
        TableHash th;
        cudaError_t e = cudaSuccess;
        for (size_t off = 0; ok && off < total; off += kIoChunk) {
            const size_t n = std::min(kIoChunk, total - off);
            e = cudaMemcpy(buf.data(), static_cast<const char *>(k->d_table) + off, n, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) break;
            th.add(buf.data(), n);
            ok = std::fwrite(buf.data(), 1, n, f) == n;
        }
        if (ok && e == cudaSuccess) {
            Writer t;
            t.u64(th.h);
            ok = std::fwrite(t.b.data(), 1, 8, f) == 8;
        }
        const int cl = std::fclose(f);
        if (e != cudaSuccess) return aw_set_error(AW_ECUDA, "table copy: %s", cudaGetErrorString(e));
        if (!ok || cl != 0) return aw_set_error(AW_EINVAL, "write to '%s' failed", path);
        return AW_OK;
    } catch (const std::bad_alloc &) {
        return aw_set_error(AW_ENOMEM, "host allocation failed");
    } catch (...) {
        return aw_set_error(AW_EINVAL, "unexpected C++ exception");
    }
}

extern "C" int aw_kernel_set_load(aw_ctx *ctx, const char *path, aw_kernel_set **out) {
    FILE *f = nullptr;
    aw_kernel_set *k = nullptr;
    auto fail = [&](int rc) {
        if (f) std::fclose(f);
        if (k) aw_kernel_set_destroy(k);
        return rc;
    };
    try {
        if (!ctx || !path || !out) return aw_set_error(AW_EINVAL, "NULL argument");
        *out = nullptr;
        f = std::fopen(path, "rb");
        if (!f) return aw_set_error(AW_EINVAL, "cannot open '%s'", path);
        // header: read a generous prefix, decode, then check its hash
        std::vector<unsigned char> head(1 << 20);
        const size_t got = std::fread(head.data(), 1, head.size(), f);
        head.resize(got);
        if (got < 16 || std::memcmp(head.data(), kSetMagic, 8) != 0)
            return fail(aw_set_error(AW_EINVAL, "'%s' is not a kernel-set file", path));
        Reader r(head);
        r.pos = 8;
        DecodedSpec d;
        if (!decode_spec(r, d)) return fail(aw_set_error(AW_EINVAL, "'%s': bad spec", path));
        const float scale = r.f32();
        const int32_t nrej = r.i32();
        const int64_t total = r.i64();
        const int32_t eb = r.i32();
        const size_t hlen = r.pos;
        const uint64_t hsum = r.u64();
        if (!r.ok || hsum != fnv1a(head.data(), hlen))
            return fail(aw_set_error(AW_EINVAL, "'%s': header checksum mismatch", path));
        AW_CUDA_TRY(cudaSetDevice(ctx->device));
        k = new aw_kernel_set();
        k->device = ctx->device;
        int rc = aw_kernel_set_geometry(&d.sp, k);
        if (rc) return fail(rc);
        if (k->total_elems != total || k->elem_bytes != eb)
            return fail(aw_set_error(AW_EINVAL, "'%s': table size does not match its spec", path));
        rc = aw_kernel_set_alloc(k);
        if (rc) return fail(rc);
        k->scale = scale;
        k->n_rejected = nrej;
        if (std::fseek(f, (long)r.pos, SEEK_SET) != 0)
            return fail(aw_set_error(AW_EINVAL, "'%s': seek failed", path));
        const size_t bytes = (size_t)total * (size_t)eb;
        std::vector<unsigned char> buf(std::min(bytes, kIoChunk) + 8);
        TableHash th;
        for (size_t off = 0; off < bytes; off += kIoChunk) {
            const size_t n = std::min(kIoChunk, bytes - off);
            if (std::fread(buf.data(), 1, n, f) != n) return fail(aw_set_error(AW_EINVAL, "'%s': truncated", path));
            th.add(buf.data(), n);
            const cudaError_t e = cudaMemcpy(static_cast<char *>(k->d_table) + off, buf.data(), n,
                                             cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return fail(aw_set_error(AW_ECUDA, "table upload: %s", cudaGetErrorString(e)));
        }
        unsigned char tail[9];
        const size_t nt = std::fread(tail, 1, 9, f);
        if (nt != 8) return fail(aw_set_error(AW_EINVAL, "'%s': %s", path, nt < 8 ? "truncated" : "trailing bytes"));
        std::vector<unsigned char> tv(tail, tail + 8);
        Reader tr(tv);
        if (tr.u64() != th.h) return fail(aw_set_error(AW_EINVAL, "'%s': table checksum mismatch", path));
        std::fclose(f);
        f = nullptr;
        *out = k;
        return AW_OK;
    } catch (const std::bad_alloc &) {
        return fail(aw_set_error(AW_ENOMEM, "host allocation failed"));
    } catch (...) {
        return fail(aw_set_error(AW_EINVAL, "unexpected C++ exception"));
    }
}

extern "C" int aw_surrogate_create(aw_ctx *ctx, const aw_surrogate_cfg *cfg, aw_surrogate **out);
extern "C" int aw_surrogate_destroy(aw_surrogate *s);

extern "C" int aw_surrogate_save(const aw_surrogate *s, const char *path) {
    try {
        if (!s || !path) return aw_set_error(AW_EINVAL, "NULL argument");
        AW_CUDA_TRY(cudaSetDevice(s->device));
        AW_CUDA_TRY(cudaDeviceSynchronize());
        std::vector<float> p((size_t)s->nparam);
        AW_CUDA_TRY(cudaMemcpy(p.data(), s->d_p, sizeof(float) * p.size(), cudaMemcpyDeviceToHost));
        Writer w;
        w.raw(kMagic, 8);
        w.i32(s->cfg.npol);
        w.i32(s->cfg.width);
        w.i32(s->cfg.n_hidden);
        w.i32((int32_t)s->norm.size());
        w.i32(s->engine);
        w.i32(s->freq_mode);
        w.f32(s->cfg.omega0);
        w.f32(s->cfg.out_scale);
        w.f64(s->cfg.D);
        w.f64(s->cfg.w_max);
        w.f64(s->cfg.f_c);
        w.f64(s->cfg.f_h);
        w.f64(s->cfg.chi_c);
        w.f64(s->cfg.chi_h);
        w.u64(s->cfg.seed);
        for (int32_t v : s->norm) w.i32(v);
        w.i64(s->nparam);
        for (float v : p) w.f32(v);
        w.i32((int32_t)s->plane_rejected.size());
        for (uint8_t v : s->plane_rejected) w.b.push_back(v);
        w.u64(fnv1a(w.b.data(), w.b.size()));
        FILE *f = std::fopen(path, "wb");
        if (!f) return aw_set_error(AW_EINVAL, "cannot open '%s' for writing", path);
        const size_t n = std::fwrite(w.b.data(), 1, w.b.size(), f);
        const int cl = std::fclose(f);
        if (n != w.b.size() || cl != 0) return aw_set_error(AW_EINVAL, "write to '%s' failed", path);
        return AW_OK;
    } catch (const std::bad_alloc &) {
        return aw_set_error(AW_ENOMEM, "host allocation failed");
    } catch (...) {
        return aw_set_error(AW_EINVAL, "unexpected C++ exception");
    }
}

extern "C" int aw_surrogate_load(aw_ctx *ctx, const char *path, aw_surrogate **out) {
    try {
        if (!ctx || !path || !out) return aw_set_error(AW_EINVAL, "NULL argument");
        *out = nullptr;
        FILE *f = std::fopen(path, "rb");
        if (!f) return aw_set_error(AW_EINVAL, "cannot open '%s'", path);
        std::vector<unsigned char> buf;
        unsigned char tmp[65536];
        size_t n;
        while ((n = std::fread(tmp, 1, sizeof(tmp), f)) > 0) buf.insert(buf.end(), tmp, tmp + n);
        const bool err = std::ferror(f) != 0;
        std::fclose(f);
        if (err) return aw_set_error(AW_EINVAL, "read of '%s' failed", path);
        if (buf.size() < 16 || std::memcmp(buf.data(), kMagic, 8) != 0)
            return aw_set_error(AW_EINVAL, "'%s' is not a surrogate file", path);
        {
            Reader tail(buf);
            tail.pos = buf.size() - 8;
            if (tail.u64() != fnv1a(buf.data(), buf.size() - 8))
                return aw_set_error(AW_EINVAL, "'%s': checksum mismatch", path);
        }
        Reader r(buf);
        r.pos = 8;
        aw_surrogate_cfg cfg{};
        cfg.npol = r.i32();
        cfg.width = r.i32();
        cfg.n_hidden = r.i32();
        cfg.norm_nw = r.i32();
        const int32_t engine = r.i32();
        const int32_t freq_mode = r.i32();
        cfg.omega0 = r.f32();
        cfg.out_scale = r.f32();
        cfg.D = r.f64();
        cfg.w_max = r.f64();
        cfg.f_c = r.f64();
        cfg.f_h = r.f64();
        cfg.chi_c = r.f64();
        cfg.chi_h = r.f64();
        cfg.seed = r.u64();
        if (!r.ok || cfg.norm_nw < 1 || cfg.norm_nw > 256)
            return aw_set_error(AW_EINVAL, "'%s': bad header", path);
        std::vector<int32_t> norm((size_t)cfg.norm_nw);
        for (auto &v : norm) v = r.i32();
        cfg.norm_supports = norm.data();
        const int64_t nparam = r.i64();
        if (!r.ok || nparam < 1 || nparam > (int64_t)(buf.size() / 4))
            return aw_set_error(AW_EINVAL, "'%s': bad parameter count", path);
        std::vector<float> p((size_t)nparam);
        for (auto &v : p) v = r.f32();
        const int32_t nrej = r.i32();
        if (!r.ok || nrej < 0 || nrej > 256 || !r.need((size_t)nrej))
            return aw_set_error(AW_EINVAL, "'%s': truncated", path);
        std::vector<uint8_t> rej(buf.begin() + (long)r.pos, buf.begin() + (long)r.pos + nrej);
        r.pos += (size_t)nrej;
        if (r.pos != buf.size() - 8) return aw_set_error(AW_EINVAL, "'%s': trailing bytes", path);
        if (engine != AW_ENGINE_MMA_SYNC && engine != AW_ENGINE_TCGEN05)
            return aw_set_error(AW_EINVAL, "'%s': engine %d", path, engine);
        if (freq_mode != AW_FREQ_BIN && freq_mode != AW_FREQ_CHANNEL)
            return aw_set_error(AW_EINVAL, "'%s': frequency mode %d", path, freq_mode);
        aw_surrogate *s = nullptr;
        int rc = aw_surrogate_create(ctx, &cfg, &s);
        if (rc) return rc;
        if (s->nparam != nparam) {
            aw_surrogate_destroy(s);
            return aw_set_error(AW_EINVAL, "'%s': %lld parameters, the configuration has %lld", path,
                                (long long)nparam, (long long)s->nparam);
        }
        cudaError_t e = cudaMemcpy(s->d_p, p.data(), sizeof(float) * p.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) rc = aw_sur_sync_half(s, 0);
        if (e == cudaSuccess && rc == AW_OK) e = cudaDeviceSynchronize();
        if (e != cudaSuccess || rc != AW_OK) {
            aw_surrogate_destroy(s);
            return rc ? rc : aw_set_error(AW_ECUDA, "surrogate upload: %s", cudaGetErrorString(e));
        }
        s->plane_rejected = rej;
        s->engine = engine;
        s->freq_mode = freq_mode;
        *out = s;
        return AW_OK;
    } catch (const std::bad_alloc &) {
        return aw_set_error(AW_ENOMEM, "host allocation failed");
    } catch (...) {
        return aw_set_error(AW_EINVAL, "unexpected C++ exception");
    }
}
