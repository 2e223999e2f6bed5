// aw_surrogate_save / aw_surrogate_load: the surrogate's configuration,
// FP32 parameters, per-w-plane rejection state and engine in one file.
//
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
