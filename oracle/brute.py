"""Pure-Python brute force of Eq. 3 for tiny inputs (N <= 4, tens of events).

TEST INFRASTRUCTURE. Python complex numbers and explicit loops, written from
the equation without any rearrangement: the data term keeps the paper's
double sum over (alpha, alpha'), and the MC bracket is summed per entry.
It exists to pin the C oracle, not to be fast.
"""
import cmath
import math


def nll(A, A_mc, n_gen, V):
    """-ln L of Eq. 3: A, A_mc are lists of per-event lists of complex amplitudes."""
    N = len(V)
    data = 0.0
    for amp in A:
        s = 0j
        for a in range(N):
            for b in range(N):
                s += V[a] * V[b].conjugate() * amp[a] * amp[b].conjugate()
        data -= math.log(s.real)
    norm = 0j
    for a in range(N):
        for b in range(N):
            bracket = 0j
            for amp in A_mc:
                bracket += amp[a] * amp[b].conjugate()
            norm += V[a] * V[b].conjugate() * bracket / n_gen
    return data + norm.real


def norm_matrix(A_mc, n_gen, N):
    """M[a][b] = (1/N_gen) sum_j conj(A_a(j)) A_b(j)."""
    return [[sum(amp[a].conjugate() * amp[b] for amp in A_mc) / n_gen for b in range(N)]
            for a in range(N)]


def wirtinger_grad(A, A_mc, n_gen, V, h=1e-6):
    """dNLL/dV*_a = (dNLL/dRe V_a + i dNLL/dIm V_a) / 2, by central differences
    of the brute-force NLL."""
    out = []
    for a in range(len(V)):
        parts = []
        for step in (h, 1j * h):
            vp = list(V)
            vm = list(V)
            vp[a] += step
            vm[a] -= step
            parts.append((nll(A, A_mc, n_gen, vp) - nll(A, A_mc, n_gen, vm)) / (2 * h))
        out.append(complex(parts[0], parts[1]) / 2)
    return out


def grad_closed(A, A_mc, n_gen, V):
    """The Wirtinger gradient written out per term:
    g_a = -sum_i conj(A_ia) S_i / |S_i|^2 + (1/N_gen) sum_j conj(A_ja) S_j."""
    N = len(V)
    g = [0j] * N
    for amp in A:
        s = sum(V[b] * amp[b] for b in range(N))
        for a in range(N):
            g[a] -= amp[a].conjugate() * s / (abs(s) ** 2)
    for amp in A_mc:
        s = sum(V[b] * amp[b] for b in range(N))
        for a in range(N):
            g[a] += amp[a].conjugate() * s / n_gen
    return g


def rotate(V, phi):
    return [v * cmath.exp(1j * phi) for v in V]


def nll_incoh(A, A_mc, n_gen, V):
    """-ln L of Eq. 3 with the per-event products summed over incoherent
    components: A, A_mc are lists (events) of lists (components) of lists
    (waves) of complex amplitudes."""
    N = len(V)
    data = 0.0
    for comps in A:
        s = 0j
        for amp in comps:
            for a in range(N):
                for b in range(N):
                    s += V[a] * V[b].conjugate() * amp[a] * amp[b].conjugate()
        data -= math.log(s.real)
    norm = 0j
    for a in range(N):
        for b in range(N):
            bracket = 0j
            for comps in A_mc:
                for amp in comps:
                    bracket += amp[a] * amp[b].conjugate()
            norm += V[a] * V[b].conjugate() * bracket / n_gen
    return data + norm.real


def wirtinger_grad_incoh(A, A_mc, n_gen, V, h=1e-6):
    """Central differences of nll_incoh, combined as in wirtinger_grad."""
    out = []
    for a in range(len(V)):
        parts = []
        for step in (h, 1j * h):
            vp = list(V)
            vm = list(V)
            vp[a] += step
            vm[a] -= step
            parts.append((nll_incoh(A, A_mc, n_gen, vp) - nll_incoh(A, A_mc, n_gen, vm)) / (2 * h))
        out.append(complex(parts[0], parts[1]) / 2)
    return out
