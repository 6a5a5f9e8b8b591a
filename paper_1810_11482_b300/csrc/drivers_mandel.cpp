// Sec. 5.1.3: Mandelbrot images written to PNG files, either synchronously
// after each image or as a continuation on the worker pool, so that the
// host encodes and writes one image while the device computes the next
// (the paper's hpx::async write).
//
// The PNG writer is a plain streaming encoder: 8-bit RGB, no interlace,
// filter type 0 on every row, the zlib stream cut into IDAT chunks of at
// most 1 MiB, CRC-32 over each chunk's type and data.
#include <zlib.h>

#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "drivers_util.hpp"
#include "runtime.hpp"

using namespace hxc;

namespace {

void put_be32(uint8_t *p, uint32_t v) {
    p[0] = (uint8_t)(v >> 24);
    p[1] = (uint8_t)(v >> 16);
    p[2] = (uint8_t)(v >> 8);
    p[3] = (uint8_t)v;
}

bool write_chunk(FILE *f, const char *type, const uint8_t *data, size_t n) {
    uint8_t hdr[8];
    put_be32(hdr, (uint32_t)n);
    memcpy(hdr + 4, type, 4);
    uLong crc = crc32(0L, reinterpret_cast<const Bytef *>(type), 4);
    if (n) crc = crc32(crc, data, (uInt)n);
    uint8_t tail[4];
    put_be32(tail, (uint32_t)crc);
    return fwrite(hdr, 1, 8, f) == 8 && (n == 0 || fwrite(data, 1, n, f) == n) &&
           fwrite(tail, 1, 4, f) == 4;
}

hxc_status png_write(const uint8_t *rgb, int64_t width, int64_t height, int level,
                     const std::string &path) {
    FILE *f = fopen(path.c_str(), "wb");
    if (!f) {
        set_error("png: cannot open %s for writing", path.c_str());
        return HXC_E_INVALID;
    }
    static const uint8_t sig[8] = {0x89, 'P', 'N', 'G', 0x0D, 0x0A, 0x1A, 0x0A};
    uint8_t ihdr[13];
    put_be32(ihdr, (uint32_t)width);
    put_be32(ihdr + 4, (uint32_t)height);
    ihdr[8] = 8;   // bits per sample
    ihdr[9] = 2;   // truecolour
    ihdr[10] = 0;  // deflate
    ihdr[11] = 0;  // adaptive filtering (each row names its filter)
    ihdr[12] = 0;  // no interlace
    bool ok = fwrite(sig, 1, 8, f) == 8 && write_chunk(f, "IHDR", ihdr, 13);
    z_stream z;
    memset(&z, 0, sizeof z);
    ok = ok && deflateInit(&z, level) == Z_OK;
    std::vector<uint8_t> out(1 << 20);
    const size_t row = (size_t)width * 3;
    static const uint8_t filter_none = 0;
    auto pump = [&](const uint8_t *src, size_t n, int flush) {
        z.next_in = const_cast<Bytef *>(src);
        z.avail_in = (uInt)n;
        do {
            z.next_out = out.data();
            z.avail_out = (uInt)out.size();
            int r = deflate(&z, flush);
            if (r == Z_STREAM_ERROR) return false;
            size_t have = out.size() - z.avail_out;
            if (have && !write_chunk(f, "IDAT", out.data(), have)) return false;
        } while (z.avail_out == 0 || (flush == Z_FINISH && z.avail_in != 0));
        return true;
    };
    for (int64_t j = 0; ok && j < height; j++)
        ok = pump(&filter_none, 1, Z_NO_FLUSH) && pump(rgb + (size_t)j * row, row, Z_NO_FLUSH);
    ok = ok && pump(nullptr, 0, Z_FINISH);
    deflateEnd(&z);
    ok = ok && write_chunk(f, "IEND", nullptr, 0);
    ok = (fclose(f) == 0) && ok;
    if (!ok) {
        set_error("png: writing %s failed", path.c_str());
        return HXC_E_INVALID;
    }
    return HXC_OK;
}

}  // namespace

extern "C" {

hxc_status hxc_png_write(const uint8_t *rgb, int64_t width, int64_t height, int level,
                         const char *path) {
    if (!rgb || !path || width < 1 || height < 1 || width > 0x7fffffff || height > 0x7fffffff ||
        level < -1 || level > 9) {
        set_error("hxc_png_write: need an image, a path, 1 <= width, height < 2^31, level -1..9");
        return HXC_E_INVALID;
    }
    return png_write(rgb, width, height, level, path);
}

hxc_status hxc_mandelbrot_png(hxc_device dh, const hxc_mandelbrot_args *args, uint8_t *host_rgb,
                              const char *path, int level, int async_write, int slot,
                              const hxc_future *deps, int ndeps, hxc_future *out) {
    hxc::drv::NvtxRange nvtx_range("hxc_mandelbrot_png");
    if (!args || !host_rgb || !path || !out || level < -1 || level > 9 || args->width < 1 ||
        args->height < 1) {
        set_error("hxc_mandelbrot_png: NULL or invalid argument");
        return HXC_E_INVALID;
    }
    const int64_t w = args->width, h = args->height;
    hxc_future kf = nullptr, rf = nullptr;
    hxc_status st = hxc_launch(dh, HXC_K_MANDELBROT, args, sizeof *args, nullptr, slot, deps, ndeps,
                               &kf);
    if (st) return st;
    st = hxc_buffer_enqueue_read(args->rgb, 0, (size_t)w * h * 3, host_rgb, slot, &kf, 1, &rf);
    hxc_future_release(kf);
    if (st) return st;
    const std::string p = path;
    if (!async_write) {
        st = hxc_future_wait(rf, -1);
        hxc_future_release(rf);
        if (!st) st = png_write(host_rgb, w, h, level, p);
        *out = to_handle(make_done(st));
        return st;
    }
    FutRef image = fut_from_handle(rf);
    hxc_future_release(rf);
    FutRef done = make_pending();
    fut_on_done(image, [done, host_rgb, w, h, level, p](hxc_status s) {
        if (s != HXC_OK) {
            fut_set_done(done, HXC_E_DEP_FAILED);
            return;
        }
        pool().submit([done, host_rgb, w, h, level, p] {
            fut_set_done(done, png_write(host_rgb, w, h, level, p));
        });
    });
    *out = to_handle(done);
    return HXC_OK;
}

}  // extern "C"
