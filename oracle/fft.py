"""Oracle DFT: a plain recursive mixed-radix Cooley--Tukey transform.

Test infrastructure only (see ``oracle/__init__``).

Definition (the transform behind the "Fourier pseudospectral discretization",
Sec. 4.1): for a length-n sequence x_j,

    forward   X_m = sum_j x_j exp(-2 pi i m j / n)
    inverse   x_j = (1/n) sum_m X_m exp(+2 pi i m j / n)

The fast routine below is decimation in time: split x into p interleaved
subsequences x[r::p] (p the smallest prime factor of n), transform each, and
recombine with X_m = sum_r exp(-2 pi i r m / n) * S_r[m mod (n/p)]. Lengths
whose smallest prime factor is the length itself are done by the O(n^2) sum.
``dft_direct`` is that O(n^2) sum for any n and is the pin for the fast path.
"""
import numpy as np


def _smallest_prime_factor(n):
    p = 2
    while p * p <= n:
        if n % p == 0:
            return p
        p += 1
    return n


def dft_direct(x, sign=-1, axis=-1):
    """O(n^2) DFT along ``axis`` straight from the definition (no scaling)."""
    x = np.moveaxis(np.asarray(x, dtype=np.complex128), axis, -1)
    n = x.shape[-1]
    j = np.arange(n)
    w = np.exp(sign * 2j * np.pi * np.outer(j, j) / n)
    return np.moveaxis(x @ w.T, -1, axis)


def _fft_last(x, sign):
    n = x.shape[-1]
    if n == 1:
        return x.copy()
    p = _smallest_prime_factor(n)
    if p == n:
        return dft_direct(x, sign, axis=-1)
    m = n // p
    subs = [_fft_last(x[..., r::p], sign) for r in range(p)]
    k = np.arange(n)
    out = np.zeros(x.shape, dtype=np.complex128)
    for r in range(p):
        twiddle = np.exp(sign * 2j * np.pi * r * k / n)
        out += twiddle * subs[r][..., k % m]
    return out


def fft(x, axis=-1):
    """Forward DFT along one axis (no scaling)."""
    x = np.moveaxis(np.asarray(x, dtype=np.complex128), axis, -1)
    return np.moveaxis(_fft_last(x, -1), -1, axis)


def ifft(x, axis=-1):
    """Inverse DFT along one axis, including the 1/n factor."""
    x = np.moveaxis(np.asarray(x, dtype=np.complex128), axis, -1)
    n = x.shape[-1]
    return np.moveaxis(_fft_last(x, +1) / n, -1, axis)


def fftn3(u):
    """Full complex 3D forward DFT over the last three axes."""
    return fft(fft(fft(u, -1), -2), -3)


def ifftn3(U):
    """Full complex 3D inverse DFT over the last three axes (1/n^3 included)."""
    return ifft(ifft(ifft(U, -3), -2), -1)


def rfft3(u):
    """Forward 3D DFT of a real field, kept on the half spectrum kz = 0..n/2.

    Layout: ``u[..., ix, iy, iz]`` -> ``U[..., kx, ky, kz]`` (kz = 0..n/2).
    """
    n = u.shape[-1]
    return fftn3(u)[..., : n // 2 + 1]


def irfft3(U, n):
    """Inverse of ``rfft3`` (n points along z; the x and y sizes are U's):
    rebuild the full Hermitian spectrum, transform back.

    The missing kz = n/2+1..n-1 planes come from X(-k) = conj(X(k)); the
    result's imaginary part is dropped (it is zero up to rounding for a
    Hermitian spectrum).
    """
    U = np.asarray(U, dtype=np.complex128)
    full = np.zeros(U.shape[:-1] + (n,), dtype=np.complex128)
    full[..., : n // 2 + 1] = U
    negx = (-np.arange(U.shape[-3])) % U.shape[-3]
    negy = (-np.arange(U.shape[-2])) % U.shape[-2]
    for kz in range(n // 2 + 1, n):
        # X[kx, ky, kz] = conj(X[-kx, -ky, n-kz])
        src = U[..., :, :, n - kz]
        full[..., :, :, kz] = np.conj(src[..., negx, :][..., :, negy])
    return ifftn3(full).real
