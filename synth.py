"""Seeded synthetic inputs shaped like the paper's experiments (Section 7).

Shared by the tests, smoke() and bench.py for BOTH the CUDA path and the CPU
oracle; it holds none of the solver's arithmetic, only input construction:

    A = U diag(sigma) V^*                      (Eq. matrix_definition)
    U: Q factor of an m x m matrix of i.i.d. (N(0,1) + i N(0,1))/sqrt(2)
    V: Q factor of an n x m matrix of the same entries
    sigma_j = 10^(-e (j-1)/(m-1)), j = 1..m    (the paper uses e = 6, kappa = 1e6)
    b: i.i.d. complex Gaussian (the workloads' right-hand side), or the
       paper's b = A p with p = m^{-1/2} sum_j eps_j v_j, eps_j = +-1
       (Eqs. rhs_definition, exact_solution).

Householder QR replaces the paper's Gram-Schmidt; the two give the same
orthonormal factors up to a unit phase per column. Random numbers come from
numpy's PCG64 seeded with `seed`; large factorisations may run on a torch
device (input construction only), the draws always come from numpy.
"""
import numpy as np


def _gauss(rng, shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)


def _orth(G, device):
    if device is None or device == "cpu":
        Q, _ = np.linalg.qr(G)
        return Q
    import torch
    Q, _ = torch.linalg.qr(torch.from_numpy(G).to(device))
    return Q


def sigmas(m, exponent):
    if m == 1:
        return np.ones(1)
    return 10.0 ** (-exponent * np.arange(m) / (m - 1))


class System:
    """One synthetic system; arrays are numpy (device=None/'cpu') or torch tensors."""

    def __init__(self, A, b, U=None, sigma=None, V=None, p=None):
        self.A, self.b, self.U, self.sigma, self.V, self.p = A, b, U, sigma, V, p


def make_system(m, n, exponent, seed, dtype="c128", rhs="gaussian", nrhs=1,
                device=None, keep_factors=False, cache_dir=None):
    """A (m x n, row-major, complex128 or complex64 storage) and b (m, or m x nrhs).

    rhs: "gaussian" (the workloads) or "paper" (b = A p, p = sum eps_j v_j / sqrt(m)).
    device: None/"cpu" builds with numpy; "cuda"/"cuda:0" builds the factors
    with torch on that device and returns torch tensors there.
    cache_dir: if given, A and b are stored there as .npy files after the first
    build and loaded on later calls with the same arguments.
    """
    if cache_dir is not None and not keep_factors:
        import os
        key = "sys_%d_%d_%g_%d_%s_%s_%d" % (m, n, exponent, seed, dtype, rhs, nrhs)
        fa, fb = os.path.join(cache_dir, key + "_A.npy"), os.path.join(cache_dir, key + "_b.npy")
        if os.path.exists(fa) and os.path.exists(fb):
            A, b = np.load(fa), np.load(fb)
            if device is not None and device != "cpu":
                import torch
                return System(torch.from_numpy(A).to(device), torch.from_numpy(b).to(device))
            return System(A, b)
        sysm = make_system(m, n, exponent, seed, dtype, rhs, nrhs, device)
        os.makedirs(cache_dir, exist_ok=True)
        A = sysm.A if isinstance(sysm.A, np.ndarray) else sysm.A.cpu().numpy()
        b = sysm.b if isinstance(sysm.b, np.ndarray) else sysm.b.cpu().numpy()
        np.save(fa + ".tmp.npy", A)
        np.save(fb + ".tmp.npy", b)
        os.replace(fa + ".tmp.npy", fa)
        os.replace(fb + ".tmp.npy", fb)
        return sysm
    rng = np.random.default_rng(seed)
    Gu = _gauss(rng, (m, m))
    Gv = _gauss(rng, (n, m))
    U = _orth(Gu, device)
    V = _orth(Gv, device)
    sig = sigmas(m, exponent)
    p = None
    if device is None or device == "cpu":
        A = (U * sig[None, :]) @ V.conj().T
        if rhs == "paper":
            eps = np.where(rng.random(m) < 0.5, -1.0, 1.0)
            p = (V @ eps) / np.sqrt(m)
            b = A @ p
        else:
            b = _gauss(rng, (m, nrhs) if nrhs > 1 else (m,))
        if dtype == "c64":
            A = A.astype(np.complex64)
        A = np.ascontiguousarray(A)
    else:
        import torch
        s = torch.from_numpy(sig).to(device=device, dtype=torch.float64)
        A = (U * s[None, :]) @ V.conj().T
        if rhs == "paper":
            eps = np.where(rng.random(m) < 0.5, -1.0, 1.0)
            pt = (V @ torch.from_numpy(eps + 0j).to(device)) / np.sqrt(m)
            b = A @ pt
            p = pt
        else:
            b = torch.from_numpy(_gauss(rng, (m, nrhs) if nrhs > 1 else (m,))).to(device)
        if dtype == "c64":
            A = A.to(torch.complex64)
        A = A.contiguous()
    sysm = System(A, b, p=p)
    if keep_factors:
        sysm.U, sysm.sigma, sysm.V = U, sig, V
    return sysm


# The five workloads (sizes and spectra) the library is exercised on.
WORKLOADS = {
    "c1_plain_64x1024": dict(m=64, n=1024, exponent=3, dtype="c128", eps=1e-12, seed=1001),
    "c2_plain_512x65536": dict(m=512, n=65536, exponent=6, dtype="c128", eps=1e-12, seed=1002),
    "c3_precision_2048x262144": dict(m=2048, n=262144, exponent=5, dtype="c64", eps=1e-10, seed=1003),
    "c5_blockrhs_4096x131072": dict(m=4096, n=131072, exponent=6, dtype="c64", eps=1e-10, seed=1005,
                                    nrhs=64),
}


def batch_shapes(count=256, seed=4000):
    """The batching workload: m uniform in [32, 512], n = m k with k uniform in [8, 64]."""
    rng = np.random.default_rng(seed)
    ms = rng.integers(32, 513, size=count)
    ks = rng.integers(8, 65, size=count)
    return [(int(a), int(a * k)) for a, k in zip(ms, ks)]
