"""Work and traffic model of one FA-SD iteration, per lattice site.

Used by bench.py to turn measured kernel times into roofline fractions.

Bytes: the algorithmic (compulsory) traffic of each kernel of the schedule
(pass A, pass B, pass C + g, update, measure): every field a kernel needs is
counted once, neighbour re-reads are not.

FP64 work: instructions issued to the FP64 pipe (FMA, MUL and ADD each count
one), counted from the formulation each kernel uses:
  * radix-R DFT butterflies: R=2: 4, R=3: 14, R=4: 16, R=8: 56 operations;
    R-1 complex twiddle products (4 operations each) for every butterfly
    with a non-zero twiddle index;
  * complex product 4, complex multiply-add 4, third row (a x b)^* 24;
  * g = reunitarize(1 + Delta'): 64 for rows 1-2 (two rsqrt counted as 6
    each), 24 for row 3.

Loads/stores per thread in the paper's Table 1 convention (reals moved by
one thread of kernels k2, k5, k6) are reproduced by ``table1_counts``.
"""

from __future__ import annotations

KERNELS = ("pass_A", "pass_B", "pass_C", "update", "measure")

DFT_OPS = {2: 4, 3: 14, 4: 16, 8: 56}


def radix_schedule(N: int) -> list[int]:
    a = b = 0
    n = N
    while n % 2 == 0:
        n //= 2
        a += 1
    while n % 3 == 0:
        n //= 3
        b += 1
    if n != 1 or N < 2:
        raise ValueError(f"extent {N} is not 2^a 3^b")
    r = [8] * (a // 3)
    if a % 3 == 2:
        r.append(4)
    if a % 3 == 1:
        r.append(2)
    return r + [3] * b


def fft1d_ops_per_point(N: int) -> float:
    """FP64 operations per point of one length-N transform of the schedule."""
    ops = 0.0
    Ns = 1
    for R in radix_schedule(N):
        nb = N // R
        tw_frac = (Ns - 1) / Ns  # butterflies with a non-zero twiddle index
        ops += nb * (DFT_OPS[R] + (R - 1) * 4 * tw_frac)
        Ns *= R
    return ops / N


def fp64_ops_per_site(extents, rows: int = 3, track_G: bool = False,
                      decomposition: str = "2d2d") -> dict[str, float]:
    """FP64-pipe operations per site of every kernel of the FP64 body.

    With the 1D x 4 or 3D + 1D decompositions "pass_A" is the forward x, y, z
    transforms, "pass_B" the t pass with the filter and "pass_C" the inverse
    x, y, z transforms and g."""
    lx, ly, lz, lt = extents
    fxy = fft1d_ops_per_point(lx) + fft1d_ops_per_point(ly)
    fzt = fft1d_ops_per_point(lz) + fft1d_ops_per_point(lt)
    if decomposition != "2d2d":
        fxy = fxy + fft1d_ops_per_point(lz)
        fzt = fft1d_ops_per_point(lt)
    recon = 24 if rows == 2 else 0          # third row of a 12-real matrix
    link_update = 72 + 72 + 24              # rows 1-2 of g U, rows 1-2 of (g U) h^dag, row 3
    update = 4 * (link_update + 2 * recon)  # U and g(x+mu) rebuilt when stored as 12 reals
    per_link_measure = 18 + 15 + 2 * recon  # forward and backward link
    measure = 4 * per_link_measure + 6 + 6 + 12 + 10
    gauge = 64 + 24 + (108 if track_G else 0)
    return {
        "pass_A": 4 * fxy,
        "pass_B": 4 * (2 * fzt + 2),
        "pass_C": 4 * fxy + gauge,
        "update": update,
        "measure": measure,
    }


def fp32_path_fp64_ops_per_site() -> dict[str, float]:
    """FP64 operations of the FP32 body: only the reunitarisation (pass C) and the F/theta sums."""
    return {"pass_A": 0.0, "pass_B": 0.0, "pass_C": 64.0, "update": 0.0, "measure": 12 + 10 + 12}


def bytes_per_site(real_bytes: int, rows: int, g_rows: int, track_G: bool = False,
                   k_bytes: int | None = None, decomposition: str = "2d2d") -> dict[str, float]:
    """Compulsory DRAM bytes per site of every kernel (links and fields read/written once).

    1D x 4 moves the divergence 3 times in each of the forward and inverse
    groups; 3D + 1D once (the categories are those of ``fp64_ops_per_site``)."""
    link = 4 * rows * 3 * 2 * real_bytes      # four links
    gsz = g_rows * 3 * 2 * real_bytes
    delta = 4 * 2 * real_bytes                # four complex fields
    kb = real_bytes if k_bytes is None else k_bytes
    G = 2 * 9 * 2 * real_bytes if track_G else 0
    sweeps = 3 if decomposition == "1d4" else 1
    g_read = delta if decomposition != "2d2d" else 0   # the separate g kernel reads the field again
    return {
        "pass_A": sweeps * 2 * delta,
        "pass_B": 2 * delta + kb,
        "pass_C": (sweeps * 2 * delta + g_read if decomposition != "2d2d" else delta) + gsz + G,
        "update": 2 * link + gsz,
        "measure": link + delta,
    }


def fused_update_measure_bytes(real_bytes: int, rows: int, g_rows: int) -> int:
    """Compulsory bytes per site of the fused update + measurement: the links
    read and written once, g read once, the divergence written (the backward
    links and g(x +- mu^) are neighbour re-reads)."""
    link = 4 * rows * 3 * 2 * real_bytes
    return 2 * link + g_rows * 3 * 2 * real_bytes + 4 * 2 * real_bytes


def b_alg_per_site(real_bytes: int, rows: int) -> int:
    """B_alg = 2 (4 S_L) + 2 S_g + 4 S_Delta: links read and written once, g written
    and read once, the divergence swept four times (a fused update+measure schedule)."""
    S_L = rows * 3 * 2 * real_bytes
    S_g = S_L
    S_D = 8 * real_bytes
    return 2 * 4 * S_L + 2 * S_g + 4 * S_D


def table1_counts(rows: int) -> dict[str, tuple[int, int]]:
    """Reals loaded/stored per thread by k2, k5, k6 (the paper's Table 1 convention):
    k2 reads the 4 links at x and the 4 backward links and stores Delta(x) in the
    link storage plus the two partial sums (F and theta); k5 reads and writes one
    matrix; k6 reads 4 links, g(x) and the 4 forward g(x+mu), and writes the 4 links."""
    r = rows * 6
    return {
        "k2": (8 * r, r + 2),
        "k5": (r, r),
        "k6": (4 * r + 5 * r, 4 * r),
    }


def paper_fft_flops_per_site(extents) -> float:
    """The paper's flop count of one 2D + 2D FFT per site, 5 (log2(nx ny) + log2(nz nt))
    (Sec. 3.2, before Table 1)."""
    import math
    lx, ly, lz, lt = extents
    return 5.0 * (math.log2(lx * ly) + math.log2(lz * lt))


def or_bytes_per_site_sweep(real_bytes: int, rows: int, track_G: bool = False) -> int:
    """Compulsory DRAM bytes per site of one overrelaxation sweep: each colour
    reads and writes every link of the lattice once (the forward links of its
    own sites and the backward links of theirs), i.e. 2 x 2 x 4 S_L per site
    and sweep; G, when tracked, is read and written once per sweep."""
    S_L = rows * 3 * 2 * real_bytes
    G = 2 * 9 * 2 * real_bytes if track_G else 0
    return 2 * 2 * 4 * S_L + G


def or_ops_per_site_sweep(rows: int = 3, track_G: bool = False) -> int:
    """Floating-point instructions (lane precision; FMA, MUL, ADD one each) per
    site of one overrelaxation sweep (every site is updated once per sweep):
      * w(x): 8 links summed, 18 each, plus the third rows of 12-real links (24);
      * the Cabibbo-Marinari hit: 3 subgroups of 35 (components, two
        normalisations with rsqrt counted as 6) and the rotations of M and g,
        18 per column pair: 3 (M, first subgroup) + 3 + 3 (g) + 1 (M, second
        subgroup, one row of two columns: 10 each) -> 54 + 20 + 54 + 54;
      * the 8 link products: rows 1-2 (72) and the third row (24) each, plus
        the third rows the forward products need from 12-real links (24);
      * G <- g G: 108 when tracked."""
    recon = 24 if rows == 2 else 0
    w = 8 * (18 + recon)
    hit = 3 * 35 + 54 + 20 + 54 + 54
    products = 8 * (72 + 24) + 4 * recon
    return w + hit + products + (108 if track_G else 0)
