"""Export of the two-point results as one FITS file: the correlation, its
covariance and its distortion matrix, per bin, with the bins' mean
separations, redshift and pair counts.  This is the output the paper's
post-processing step writes for the Vega fitter (Appendix A; Section 3
describes it as a FITS file with the correlation, covariance and distortion
matrix that mimics PICCA's).

The file is written to the FITS 4.0 standard without a FITS library: an empty
primary HDU, then one binary-table extension (EXTNAME 'COR') with one row per
bin A = p * n_perp + t (the library's bin order; p indexes r_par, t r_perp):

    RP  1D       weighted mean r_par of the bin's pixel pairs [Mpc/h]
    RT  1D       weighted mean r_perp [Mpc/h]
    Z   1D       weighted mean redshift (0 where not given)
    NB  1K       pixel-pair count
    WE  1D       W_A, the sum of the pair weights (Eq. 2.4's denominator)
    DA  1D       xi_A (Eq. 2.4)
    CO  <nb>D    row A of the covariance of xi
    DM  <nb>D    row A of the distortion matrix D (Eq. 2.5: xi^_A = sum_B D_AB xi_B)

The header of the table carries the grid: RPMIN, RPMAX, RTMAX, NP, NT, and any
extra keywords the caller passes (e.g. OMEGAM of the fiducial cosmology).
Everything here is host-side formatting of arrays the library has computed.
"""
from __future__ import annotations

import gzip
import math
from typing import Dict, Mapping, Optional, Sequence, Tuple, Union

import numpy as np

BLOCK = 2880   # FITS logical record, bytes
CARD = 80      # header card, bytes

ArrayLike = Union[np.ndarray, "torch.Tensor"]  # noqa: F821


def _host(a, dtype) -> np.ndarray:
    """Array on the host (a torch tensor on any device, or anything numpy takes)."""
    if hasattr(a, "detach"):
        a = a.detach().cpu().numpy()
    return np.ascontiguousarray(np.asarray(a, dtype=dtype))


def _format_value(value) -> str:
    """Value field of a card, columns 11-30 for numbers and logicals (right-justified),
    a quoted string from column 11 otherwise (FITS 4.0, Section 4.2)."""
    if isinstance(value, (bool, np.bool_)):
        return f"{'T' if value else 'F':>20}"
    if isinstance(value, (int, np.integer)):
        return f"{int(value):>20d}"
    if isinstance(value, (float, np.floating)):
        v = float(value)
        if not math.isfinite(v):
            raise ValueError(f"FITS header values must be finite, got {v}")
        s = repr(v).upper()   # shortest round-trip form; exponent written with 'E'
        if "." not in s:      # a real always carries its decimal point
            s = s.replace("E", ".0E") if "E" in s else s + ".0"
        return f"{s:>20}"
    if isinstance(value, str):
        if any(ord(ch) < 32 or ord(ch) > 126 for ch in value):
            raise ValueError("FITS header strings must be printable ASCII")
        s = value.replace("'", "''")
        return "'" + f"{s:<8}" + "'"
    raise TypeError(f"unsupported FITS header value {value!r}")


def card(key: str, value=None, comment: str = "") -> bytes:
    """One 80-byte header card: keyword in columns 1-8, '= ' in 9-10, the value,
    then ' / comment'.  A card without a value (END) is the keyword alone."""
    if not key or len(key) > 8 or not all("A" <= ch <= "Z" or ch.isdigit() or ch in "-_" for ch in key):
        raise ValueError(f"invalid FITS keyword {key!r}")
    if value is None:
        text = f"{key:<8}"
    else:
        text = f"{key:<8}= " + _format_value(value)
        if comment:
            text += " / " + comment
    if len(text) > CARD:
        if value is not None and comment:
            text = text[:CARD]   # a comment may be cut; the value may not
        else:
            raise ValueError(f"FITS card longer than {CARD} characters: {text!r}")
    return text.ljust(CARD).encode("ascii")


def header(cards: Sequence[bytes]) -> bytes:
    """Header unit: the cards, END, then spaces to a whole number of blocks."""
    h = b"".join(cards) + card("END")
    return h + b" " * (-len(h) % BLOCK)


def _pad_data(data: bytes) -> bytes:
    return data + b"\0" * (-len(data) % BLOCK)


def cor_table(bins, xi, cov, dmat, rp, rt, nb, we, z=None) -> Tuple[np.ndarray, Dict[str, str]]:
    """Rows of the 'COR' table as a packed big-endian structured array, and the
    TFORM of each column."""
    n = bins.n_par * bins.n_perp
    cols = {
        "RP": _host(rp, np.float64), "RT": _host(rt, np.float64),
        "Z": _host(z, np.float64) if z is not None else np.zeros(n),
        "NB": _host(nb, np.int64), "WE": _host(we, np.float64), "DA": _host(xi, np.float64),
        "CO": _host(cov, np.float64), "DM": _host(dmat, np.float64),
    }
    for k in ("RP", "RT", "Z", "NB", "WE", "DA"):
        if cols[k].shape != (n,):
            raise ValueError(f"{k}: expected shape ({n},), got {cols[k].shape}")
    for k in ("CO", "DM"):
        if cols[k].shape != (n, n):
            raise ValueError(f"{k}: expected shape ({n}, {n}), got {cols[k].shape}")
    dt = np.dtype([("RP", ">f8"), ("RT", ">f8"), ("Z", ">f8"), ("NB", ">i8"), ("WE", ">f8"),
                   ("DA", ">f8"), ("CO", ">f8", (n,)), ("DM", ">f8", (n,))])
    rows = np.zeros(n, dtype=dt)
    for k in dt.names:
        rows[k] = cols[k]
    tform = {k: "1D" for k in ("RP", "RT", "Z", "WE", "DA")}
    tform["NB"] = "1K"
    tform["CO"] = tform["DM"] = f"{n}D"
    return rows, tform


def cor_bytes(bins, xi, cov, dmat, rp, rt, nb, we, z=None,
              extra: Optional[Mapping[str, object]] = None) -> bytes:
    """The whole file as bytes (primary HDU + 'COR' binary table)."""
    rows, tform = cor_table(bins, xi, cov, dmat, rp, rt, nb, we, z)
    names = rows.dtype.names
    units = {"RP": "Mpc/h", "RT": "Mpc/h"}
    primary = header([card("SIMPLE", True, "conforms to FITS standard"), card("BITPIX", 8),
                      card("NAXIS", 0), card("EXTEND", True)])
    cards = [card("XTENSION", "BINTABLE", "binary table extension"), card("BITPIX", 8),
             card("NAXIS", 2), card("NAXIS1", rows.dtype.itemsize, "bytes per row"),
             card("NAXIS2", len(rows), "rows: one per (r_par, r_perp) bin"),
             card("PCOUNT", 0), card("GCOUNT", 1), card("TFIELDS", len(names))]
    for i, k in enumerate(names, 1):
        cards.append(card(f"TTYPE{i}", k))
        cards.append(card(f"TFORM{i}", tform[k]))
        if k in units:
            cards.append(card(f"TUNIT{i}", units[k]))
    cards += [card("EXTNAME", "COR"),
              card("RPMIN", 0.0, "lower edge of r_par [Mpc/h]"),
              card("RPMAX", float(bins.r_par_max), "upper edge of r_par [Mpc/h]"),
              card("RTMAX", float(bins.r_perp_max), "upper edge of r_perp [Mpc/h]"),
              card("NP", int(bins.n_par), "r_par bins"), card("NT", int(bins.n_perp), "r_perp bins")]
    for k, v in (extra or {}).items():
        cards.append(card(k, v))
    return primary + header(cards) + _pad_data(rows.tobytes())


def write_cor(path: str, bins, xi, cov, dmat, rp, rt, nb, we, z=None,
              extra: Optional[Mapping[str, object]] = None) -> int:
    """Write the file (gzip-compressed when path ends in '.gz'); returns the
    uncompressed size in bytes.

    xi, we, rp, rt, nb, z: [n_par * n_perp] (``lya_xi``, ``lya_xi_bin_means``);
    cov: [nb, nb] (``lya_xi_covariance``); dmat: [nb, nb] (``lya_dmat``)."""
    data = cor_bytes(bins, xi, cov, dmat, rp, rt, nb, we, z, extra)
    if path.endswith(".gz"):
        with gzip.open(path, "wb") as f:
            f.write(data)
    else:
        with open(path, "wb") as f:
            f.write(data)
    return len(data)
