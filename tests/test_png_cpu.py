"""The PNG writer (hxc_png_write) on the host: the file is decoded here with
the standard library alone (chunk lengths, CRC-32 of every chunk, the zlib
stream, the row filters) and must give back the image bit for bit."""
import struct
import zlib

import numpy as np
import pytest

from paper_1810_11482_b300 import hxc, synth


def decode_png(path):
    data = open(path, "rb").read()
    assert data[:8] == b"\x89PNG\r\n\x1a\n"
    pos, chunks = 8, []
    while pos < len(data):
        (n,) = struct.unpack(">I", data[pos:pos + 4])
        kind, body = data[pos + 4:pos + 8], data[pos + 8:pos + 8 + n]
        (crc,) = struct.unpack(">I", data[pos + 8 + n:pos + 12 + n])
        assert crc == zlib.crc32(kind + body) & 0xFFFFFFFF, kind
        chunks.append((kind, body))
        pos += 12 + n
    assert chunks[0][0] == b"IHDR" and chunks[-1] == (b"IEND", b"")
    w, h, depth, ctype, comp, filt, inter = struct.unpack(">IIBBBBB", chunks[0][1])
    assert (depth, ctype, comp, filt, inter) == (8, 2, 0, 0, 0)
    raw = zlib.decompress(b"".join(b for k, b in chunks if k == b"IDAT"))
    rows = np.frombuffer(raw, dtype=np.uint8).reshape(h, 1 + 3 * w)
    assert (rows[:, 0] == 0).all()  # filter type 0 on every row
    return rows[:, 1:].reshape(h, w, 3), sum(1 for k, _ in chunks if k == b"IDAT")


@pytest.mark.parametrize("w,h,level", [(1, 1, 0), (37, 5, 6), (640, 481, 1), (1500, 900, -1)])
def test_png_roundtrip(tmp_path, w, h, level):
    img = (synth.uniform(30 + w, w * h * 3) * 256).astype(np.uint8).reshape(h, w, 3)
    img[h // 2:] = 7  # a compressible half
    path = tmp_path / "x.png"
    hxc.png_write(img, path, level)
    got, nidat = decode_png(path)
    assert np.array_equal(got, img)
    if w * h * 3 > (4 << 20):
        assert nidat > 1


def test_png_errors(tmp_path):
    img = np.zeros((4, 4, 3), dtype=np.uint8)
    with pytest.raises(hxc.HxcError):
        hxc.png_write(img, tmp_path / "no_such_dir" / "x.png")
    with pytest.raises(hxc.HxcError):
        hxc.png_write(img, tmp_path / "x.png", level=11)
