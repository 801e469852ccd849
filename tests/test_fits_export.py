"""FITS export of the two-point results (host logic, no GPU).

The file is read back here with a parser of its own (80-byte cards, 2880-byte
blocks, big-endian rows decoded from the TFORMs), and card layouts are checked
against the FITS 4.0 column rules written out by hand: keyword in columns 1-8,
'= ' in 9-10, numbers and logicals right-justified to column 30, strings quoted
from column 11 and padded to at least 8 characters.
"""
import gzip
import struct

import numpy as np
import pytest
import torch

from paper_2507_00129_gb300 import fits_export as fx
from paper_2507_00129_gb300.synth import Bins


def _card_text(key, value_field, comment=""):
    s = f"{key:<8}= {value_field}"
    if comment:
        s += " / " + comment
    return s.ljust(80).encode("ascii")


def test_card_layout_follows_the_standard_columns():
    assert fx.card("SIMPLE", True) == _card_text("SIMPLE", " " * 19 + "T")
    assert fx.card("EXTEND", False) == _card_text("EXTEND", " " * 19 + "F")
    assert fx.card("NAXIS", 0) == _card_text("NAXIS", " " * 19 + "0")
    assert fx.card("NAXIS1", 40144) == _card_text("NAXIS1", " " * 15 + "40144")
    assert fx.card("NAXIS2", -3) == _card_text("NAXIS2", " " * 18 + "-3")
    assert fx.card("EXTNAME", "COR") == _card_text("EXTNAME", "'COR     '")
    assert fx.card("TFORM7", "2500D") == _card_text("TFORM7", "'2500D   '")
    # the encoded text (quote doubled) is padded to 8, so the closing quote lands in column 20
    assert fx.card("OBSERVER", "O'Hara") == _card_text("OBSERVER", "'O''Hara '")
    assert fx.card("RPMAX", 200.0) == _card_text("RPMAX", " " * 15 + "200.0")
    assert fx.card("OMEGAM", 0.315) == _card_text("OMEGAM", " " * 15 + "0.315")
    assert fx.card("EPS", 1e-05) == _card_text("EPS", " " * 13 + "1.0E-05")
    assert fx.card("BIG", -2.5e300) == _card_text("BIG", " " * 11 + "-2.5E+300")
    assert fx.card("NP", 50, "r_par bins") == _card_text("NP", " " * 18 + "50", "r_par bins")
    assert fx.card("END") == b"END" + b" " * 77
    for c in (fx.card("A", 1.0), fx.card("LONGKEY", "x" * 60, "a long comment that gets cut")):
        assert len(c) == 80


def test_card_rejects_what_fits_cannot_hold():
    with pytest.raises(ValueError):
        fx.card("RPMAX", float("inf"))
    with pytest.raises(ValueError):
        fx.card("RPMAX", float("nan"))
    with pytest.raises(ValueError):
        fx.card("TOOLONGKEY", 1)
    with pytest.raises(ValueError):
        fx.card("lower", 1)
    with pytest.raises(ValueError):
        fx.card("NAME", "x" * 80)
    with pytest.raises(ValueError):
        fx.card("NAME", "tab\there")
    with pytest.raises(TypeError):
        fx.card("NAME", [1, 2])


def test_header_is_whole_blocks_ending_in_end():
    h = fx.header([fx.card("SIMPLE", True), fx.card("BITPIX", 8), fx.card("NAXIS", 0)])
    assert len(h) == 2880
    assert h[3 * 80:4 * 80] == b"END" + b" " * 77
    assert h[4 * 80:] == b" " * (2880 - 4 * 80)
    many = fx.header([fx.card(f"K{i}", i) for i in range(36)])   # 36 cards + END spill into a second block
    assert len(many) == 2 * 2880


# --- an independent reader ---------------------------------------------------

def _parse_header(buf, start):
    cards = {}
    order = []
    pos = start
    while True:
        c = buf[pos:pos + 80].decode("ascii")
        pos += 80
        key = c[:8].strip()
        if key == "END":
            break
        assert c[8:10] == "= ", c
        v = c[10:]
        if v.lstrip().startswith("'"):
            i = v.index("'")
            j = i + 1
            out = ""
            while True:
                k = v.index("'", j)
                if k + 1 < len(v) and v[k + 1] == "'":
                    out += v[j:k] + "'"
                    j = k + 2
                    continue
                out += v[j:k]
                break
            val = out.rstrip()
        else:
            field = v[:20].strip()
            assert v[20:21] in ("", " ", "/") or v[20:].strip().startswith("/"), c
            if field in ("T", "F"):
                val = field == "T"
            elif any(ch in field for ch in ".E"):
                val = float(field)
            else:
                val = int(field)
        cards[key] = val
        order.append(key)
    end = pos + (-(pos - start) % 2880)
    assert all(b == 0x20 for b in buf[pos:end])
    return cards, order, end


def _decode_rows(buf, start, hdr):
    n_fields = hdr["TFIELDS"]
    fields = []
    for i in range(1, n_fields + 1):
        tf = hdr[f"TFORM{i}"]
        rep, code = int(tf[:-1] or 1), tf[-1]
        fields.append((hdr[f"TTYPE{i}"], rep, {"D": ">d", "K": ">q", "J": ">i", "E": ">f"}[code]))
    width = sum(rep * struct.calcsize(fmt) for _, rep, fmt in fields)
    assert width == hdr["NAXIS1"]
    out = {name: [] for name, _, _ in fields}
    pos = start
    for _ in range(hdr["NAXIS2"]):
        for name, rep, fmt in fields:
            size = struct.calcsize(fmt)
            vals = struct.unpack(">" + fmt[1] * rep, buf[pos:pos + rep * size])
            out[name].append(vals if rep > 1 else vals[0])
            pos += rep * size
    return {k: np.array(v) for k, v in out.items()}, pos


def _inputs(n_par=2, n_perp=3, seed=5):
    rng = np.random.default_rng(seed)
    bins = Bins(n_par, n_perp, 8.0, 12.0)
    nb = n_par * n_perp
    a = rng.standard_normal((nb, nb))
    return bins, dict(
        xi=rng.standard_normal(nb) * 1e-3, cov=a @ a.T * 1e-8, dmat=np.eye(nb) + 0.01 * rng.standard_normal((nb, nb)),
        rp=(np.arange(nb) // n_perp + 0.5) * 4.0, rt=(np.arange(nb) % n_perp + 0.5) * 4.0,
        nb=rng.integers(0, 2**40, nb), we=rng.random(nb) * 1e6, z=2.0 + rng.random(nb))


def test_file_reads_back_exactly(tmp_path):
    bins, d = _inputs()
    path = str(tmp_path / "cf.fits")
    size = fx.write_cor(path, bins, extra={"OMEGAM": 0.315}, **d)
    buf = open(path, "rb").read()
    assert size == len(buf) and len(buf) % 2880 == 0
    prim, order, pos = _parse_header(buf, 0)
    assert order[:4] == ["SIMPLE", "BITPIX", "NAXIS", "EXTEND"]
    assert prim == {"SIMPLE": True, "BITPIX": 8, "NAXIS": 0, "EXTEND": True}
    assert pos == 2880
    hdr, order, pos = _parse_header(buf, pos)
    # the mandatory keywords of a binary table, in the mandatory order
    assert order[:8] == ["XTENSION", "BITPIX", "NAXIS", "NAXIS1", "NAXIS2", "PCOUNT", "GCOUNT", "TFIELDS"]
    assert hdr["XTENSION"] == "BINTABLE" and hdr["BITPIX"] == 8 and hdr["NAXIS"] == 2
    assert hdr["PCOUNT"] == 0 and hdr["GCOUNT"] == 1 and hdr["EXTNAME"] == "COR"
    nb = 6
    assert hdr["NAXIS2"] == nb and hdr["NAXIS1"] == 6 * 8 + 2 * nb * 8
    assert (hdr["NP"], hdr["NT"], hdr["RPMIN"], hdr["RPMAX"], hdr["RTMAX"]) == (2, 3, 0.0, 8.0, 12.0)
    assert hdr["OMEGAM"] == 0.315
    assert [hdr[f"TTYPE{i}"] for i in range(1, 9)] == ["RP", "RT", "Z", "NB", "WE", "DA", "CO", "DM"]
    assert hdr["TFORM4"] == "1K" and hdr["TFORM7"] == "6D" and hdr["TFORM8"] == "6D"
    assert hdr["TUNIT1"] == "Mpc/h"
    rows, end = _decode_rows(buf, pos, hdr)
    for k, src in (("RP", "rp"), ("RT", "rt"), ("Z", "z"), ("NB", "nb"), ("WE", "we"), ("DA", "xi"),
                   ("CO", "cov"), ("DM", "dmat")):
        assert np.array_equal(rows[k], np.asarray(d[src])), k
    # row A holds row A of D (xi^_A = sum_B D_AB xi_B) and of the covariance
    assert np.array_equal(rows["DM"][1], d["dmat"][1])
    assert all(b == 0 for b in buf[end:]) and len(buf) - end < 2880


def test_gzip_holds_the_same_bytes(tmp_path):
    bins, d = _inputs(3, 2, seed=9)
    path = str(tmp_path / "cf.fits.gz")
    fx.write_cor(path, bins, **d)
    with gzip.open(path, "rb") as f:
        assert f.read() == fx.cor_bytes(bins, **d)


def test_torch_tensors_and_missing_z(tmp_path):
    bins, d = _inputs()
    d_t = {k: torch.from_numpy(np.asarray(v)) for k, v in d.items() if k != "z"}
    buf = fx.cor_bytes(bins, **d_t)
    _, _, pos = _parse_header(buf, 0)
    hdr, _, pos = _parse_header(buf, pos)
    rows, _ = _decode_rows(buf, pos, hdr)
    assert np.all(rows["Z"] == 0.0)
    assert np.array_equal(rows["DA"], d["xi"])


def test_shapes_are_checked():
    bins, d = _inputs()
    bad = dict(d, xi=d["xi"][:-1])
    with pytest.raises(ValueError):
        fx.cor_bytes(bins, **bad)
    bad = dict(d, dmat=d["dmat"][:, :-1])
    with pytest.raises(ValueError):
        fx.cor_bytes(bins, **bad)


def test_table_over_many_blocks(tmp_path):
    bins, d = _inputs(10, 10, seed=3)     # 100 rows of 1,648 bytes
    buf = fx.cor_bytes(bins, **d)
    _, _, pos = _parse_header(buf, 0)
    hdr, _, pos = _parse_header(buf, pos)
    assert hdr["NAXIS1"] == 48 + 2 * 100 * 8 and hdr["TFORM7"] == "100D"
    rows, end = _decode_rows(buf, pos, hdr)
    assert end - pos == 100 * 1648 and len(buf) % 2880 == 0 and len(buf) - end < 2880
    assert np.array_equal(rows["CO"], d["cov"]) and np.array_equal(rows["NB"], d["nb"])
