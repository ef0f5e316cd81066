"""RNS-CKKS scheme side of the oracle, in coefficient form, plus the graph
evaluator (neuronal firing) and the FP64 plaintext forward pass.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Shares no code with the
CUDA library.  Ciphertexts are numpy uint64 arrays c[2][L][N] holding every
residue polynomial in COEFFICIENT form; ring products go through the pinned
textbook transform (core.polymul).

arXiv 2110.13638 uses RNS-CKKS through MS-SEAL (Sec. 2.1, Sec. 3) and prints
none of the ring arithmetic; each routine is the textbook definition, with the
readings of the unspecified points stated in the docstrings:
  - keys and encryption: public-key CKKS, ternary secret, Gaussian noise;
  - relinearisation: RNS key switching with per-prime digits and one special
    prime P (digit j = residue j lifted to [0, q_j)), then ModDown by P with
    the centred remainder;
  - rescale: division by the last prime with the centred remainder;
  - the scale schedule of dense layers and of the degree-3 polynomial
    activation (Eq. sigmoid_approximate) is fixed below.
"""
import math

import numpy as np

from . import core
from .params import (prime_chain, primitive_2n_root, gauss_cdt, GAUSS_KMAX,
                     node_cost)

# sampling domains of the counter-based generator
DOM_SECRET, DOM_PK_A, DOM_PK_E, DOM_KSK_A, DOM_KSK_E = 1, 2, 3, 4, 5
DOM_ENC_U, DOM_ENC_E0, DOM_ENC_E1 = 6, 7, 8
DOM_GAL_A, DOM_GAL_E = 9, 10          # Galois (rotation) keys: object id = (k << 8) | digit
MAX_POLY_DEGREE = 31


def llround(x):
    """Round a double half away from zero to a Python int (C llround)."""
    t = math.trunc(x)
    f = x - t
    if f >= 0.5:
        return t + 1
    if f <= -0.5:
        return t - 1
    return t


def to_residue(v, q):
    """Signed integer vector -> residues mod q (uint64)."""
    v = np.asarray(v, dtype=np.int64)
    return np.mod(v, np.int64(q)).astype(np.uint64)


def centred_mod(v, p, q):
    """v: residues mod p (uint64).  Return [v_c] mod q, v_c the centred
    representative of v in (-p/2, p/2] (p odd, so (-p/2, p/2))."""
    v = np.asarray(v, dtype=np.uint64)
    half = np.uint64((p - 1) // 2)
    neg = v > half
    r = v % np.uint64(q)
    pm = np.uint64(p % q)
    # v - p mod q = r - (p mod q) mod q
    r_neg = (r + np.uint64(q) - pm) % np.uint64(q)
    return np.where(neg, r_neg, r).astype(np.uint64)


class Ciphertext:
    def __init__(self, c, level, scale):
        self.c = c            # uint64 [k][level][N], k = 2 (or 3 after a tensor)
        self.level = level
        self.scale = scale

    def copy(self):
        return Ciphertext(self.c.copy(), self.level, self.scale)


class Context:
    """Parameters and keys.  bits: coefficient-modulus bit list whose last
    entry is the special prime P (Alg. parameterise output)."""

    def __init__(self, N, bits, log_scale=40):
        self.N = N
        chain = prime_chain(N, bits)
        self.q = chain[:-1]
        self.P = chain[-1]
        self.L_top = len(self.q)
        self.key_primes = self.q + [self.P]     # residue index L_top = P
        self.psi = [primitive_2n_root(p, N) for p in self.key_primes]
        self.delta = float(2 ** log_scale)
        self.cdt = np.array(gauss_cdt(), dtype=np.uint64)
        self.seed = None

    # -- ring helpers ------------------------------------------------------
    def mul(self, a, b, r):
        """negacyclic product of two residue polynomials of key-prime index r"""
        return core.polymul(a, b, self.key_primes[r], self.psi[r])

    def _gauss(self, s0):
        return core.sample_gauss(s0, self.N, self.cdt)

    # -- keys --------------------------------------------------------------
    def keygen(self, seed):
        """Secret s (ternary), public key pk = (-a s + e, a) over the data
        primes, and relinearisation keys
            ksk_j = (-a_j s + e_j + [r == j] P s^2,  a_j)   over q_0..q_{L-1}, P
        for every data prime j (per-prime digits, one special prime)."""
        N, Lt = self.N, self.L_top
        self.seed = seed
        s = core.sample_ternary(core.stream(seed, DOM_SECRET, 0), N)
        self.s_int = s
        self.s = [to_residue(s, p) for p in self.key_primes]
        e = self._gauss(core.stream(seed, DOM_PK_E, 0))
        s_pk = core.stream(seed, DOM_PK_A, 0)
        self.pk = np.zeros((2, Lt, N), dtype=np.uint64)
        for r in range(Lt):
            q = self.q[r]
            a = core.sample_uniform(s_pk, r, q, N)
            as_ = self.mul(a, self.s[r], r)
            self.pk[0, r] = (to_residue(e, q) + (np.uint64(q) - as_) % np.uint64(q)) % np.uint64(q)
            self.pk[1, r] = a
        self.ksk = np.zeros((Lt, 2, Lt + 1, N), dtype=np.uint64)
        for j in range(Lt):
            s_a = core.stream(seed, DOM_KSK_A, j)
            e_j = self._gauss(core.stream(seed, DOM_KSK_E, j))
            for r in range(Lt + 1):
                p = self.key_primes[r]
                a = core.sample_uniform(s_a, r, p, N)
                b = (to_residue(e_j, p) + (np.uint64(p) - self.mul(a, self.s[r], r)) % np.uint64(p)) % np.uint64(p)
                if r == j:
                    s2 = self.mul(self.s[r], self.s[r], r)
                    b = (b + core.vec_mul_scalar(s2, self.P % p, p)) % np.uint64(p)
                self.ksk[j, 0, r] = b
                self.ksk[j, 1, r] = a

    # -- rotations (Galois automorphisms) ----------------------------------
    def galois_element(self, r):
        """k = 5^r mod 2N: X -> X^k moves slot j + r to slot j (rotation left
        by r); 5 has order N/2 modulo 2N, so r is taken modulo N/2."""
        return pow(5, r % (self.N // 2), 2 * self.N)

    def automorphism(self, a, k, primes):
        """a(X) -> a(X^k) mod X^N + 1 for residue rows a [len(primes)][N] in
        coefficient form: coefficient i moves to i k mod 2N, negated when that
        exponent is N or more."""
        N = self.N
        i = np.arange(N, dtype=np.int64)
        pos = (i * k) % (2 * N)
        dst = pos % N
        neg = pos >= N
        out = np.zeros_like(a)
        for r, p in enumerate(primes):
            v = a[r]
            out[r, dst] = np.where(neg, (np.uint64(p) - v) % np.uint64(p), v)
        return out

    def galois_keygen(self, k):
        """Key switching key from s(X^k) to s, in the relinearisation key's
        form with s(X^k) in place of s^2:
            gk_j = (-a_j s + e_j + [r == j] P s(X^k),  a_j)  over q_0..q_{L-1}, P"""
        N, Lt = self.N, self.L_top
        if not hasattr(self, "gk"):
            self.gk = {}
        if k in self.gk:
            return self.gk[k]
        sk = self.automorphism(np.stack([to_residue(self.s_int, p) for p in self.key_primes]), k, self.key_primes)
        gk = np.zeros((Lt, 2, Lt + 1, N), dtype=np.uint64)
        for j in range(Lt):
            s_a = core.stream(self.seed, DOM_GAL_A, (k << 8) | j)
            e_j = self._gauss(core.stream(self.seed, DOM_GAL_E, (k << 8) | j))
            for r in range(Lt + 1):
                p = self.key_primes[r]
                a = core.sample_uniform(s_a, r, p, N)
                b = (to_residue(e_j, p) + (np.uint64(p) - self.mul(a, self.s[r], r)) % np.uint64(p)) % np.uint64(p)
                if r == j:
                    b = (b + core.vec_mul_scalar(sk[r], self.P % p, p)) % np.uint64(p)
                gk[j, 0, r] = b
                gk[j, 1, r] = a
        self.gk[k] = gk
        return gk

    def rotate(self, ct, r):
        """Slots rotated left by r: (c0(X^k), c1(X^k)) with k = 5^r, then
        c1(X^k) switched from s(X^k) to s with the Galois key:
            out = (c0(X^k) + ks_0, ks_1),  ks = keyswitch(c1(X^k), gk_k)"""
        k = self.galois_element(r)
        L = ct.level
        prim = self.q[:L]
        c0 = self.automorphism(ct.c[0], k, prim)
        c1 = self.automorphism(ct.c[1], k, prim)
        ks = self.mod_down(self.keyswitch_accumulate(c1, L, self.galois_keygen(k)), L)
        c = np.empty((2, L, self.N), dtype=np.uint64)
        for t in range(L):
            q = np.uint64(self.q[t])
            c[0, t] = (c0[t] + ks[0, t]) % q
            c[1, t] = ks[1, t]
        return Ciphertext(c, L, ct.scale)

    # -- plaintext vectors (slot-wise products) ----------------------------
    def mul_plain(self, ct, m, sigma):
        """Slot-wise product with a plaintext vector: every component times
        the encoded plaintext m (int64 coefficients, scale sigma), a ring
        product in each prime."""
        c = np.empty_like(ct.c)
        for r in range(ct.level):
            mr = to_residue(m, self.q[r])
            for k in range(ct.c.shape[0]):
                c[k, r] = self.mul(ct.c[k, r], mr, r)
        return Ciphertext(c, ct.level, ct.scale * sigma)

    def add_plain(self, ct, m):
        """Slot-wise sum with a plaintext vector (encoded at the ciphertext's scale)."""
        c = ct.c.copy()
        for r in range(ct.level):
            q = np.uint64(self.q[r])
            c[0, r] = (c[0, r] + to_residue(m, self.q[r])) % q
        return Ciphertext(c, ct.level, ct.scale)

    def conv_packed(self, xs, node):
        """Kernel masquerading (Sec. 3.2) with the sum done by rotations: the
        images packed in a ciphertext (image b's pixel (i, j) at slot
        b S + i W + j) are convolved with every filter at once.  For each kernel
        position (dr, dc) the ciphertext is rotated by dr W + dc so that the
        pixel under that kernel position sits at its output slot; the merged
        mask-and-kernel vector (weight K[f, dr, dc] at the valid output slots
        b S + s r W + s c, zero elsewhere) multiplies it slot-wise; the k^2
        products are summed, rescaled, and the bias vector is added:
            y_f = rescale(sum_p rot(x, off_p) * encode(M_fp, q_{L-1})) + encode(b_f V, s_y)
        Outputs are filter-major: y[f * n + i] for input ciphertext i."""
        F, k = node["filters"], node["k"]
        M = self.N // 2
        L, s = xs[0].level, xs[0].scale
        q = float(self.q[L - 1])
        valid = packed_valid_slots(node, M)
        offs = [dr * node["W"] + dc for dr in range(k) for dc in range(k)]
        W_ = np.asarray(node["weight"], dtype=np.float64).reshape(F, k * k)
        masks = []
        for f in range(F):
            row = []
            for p in range(k * k):
                v = np.zeros(M)
                v[valid] = W_[f, p]
                row.append(self.encode(v, q))
            masks.append(row)
        out = [[None] * len(xs) for _ in range(F)]
        for i, x in enumerate(xs):
            rots = [x if o == 0 else self.rotate(x, o) for o in offs]
            for f in range(F):
                acc = None
                for p in range(k * k):
                    t = self.mul_plain(rots[p], masks[f][p], q)
                    acc = t if acc is None else self.add(acc, t)
                y = self.rescale(acc)
                bv = np.zeros(M)
                bv[valid] = float(node["bias"][f])
                out[f][i] = self.add_plain(y, self.encode(bv, y.scale))
        return [ct for row in out for ct in row]

    # -- encode / encrypt / decrypt / decode -------------------------------
    def encode(self, z, scale=None, want_frac=False):
        """Canonical-embedding encode of N/2 real slots; integer coefficients."""
        return core.encode(z, self.N, self.delta if scale is None else scale, want_frac)

    def decode(self, m, scale):
        return core.decode(m, self.N, scale)[0]

    def encrypt(self, m, ct_id, scale=None):
        """ct = (u pk0 + e0 + m, u pk1 + e1) at the top level; u ternary,
        e0/e1 Gaussian, all drawn from the stream of (seed, domain, ct_id)."""
        N, Lt = self.N, self.L_top
        u = core.sample_ternary(core.stream(self.seed, DOM_ENC_U, ct_id), N)
        e0 = self._gauss(core.stream(self.seed, DOM_ENC_E0, ct_id))
        e1 = self._gauss(core.stream(self.seed, DOM_ENC_E1, ct_id))
        c = np.zeros((2, Lt, N), dtype=np.uint64)
        for r in range(Lt):
            q = np.uint64(self.q[r])
            ur = to_residue(u, self.q[r])
            c[0, r] = (self.mul(ur, self.pk[0, r], r) + to_residue(e0, self.q[r])) % q
            c[0, r] = (c[0, r] + to_residue(m, self.q[r])) % q
            c[1, r] = (self.mul(ur, self.pk[1, r], r) + to_residue(e1, self.q[r])) % q
        return Ciphertext(c, Lt, self.delta if scale is None else scale)

    def decrypt(self, ct, check_crt=False):
        """m = c0 + c1 s, dropped to q_0, centred lift to (-q0/2, q0/2).
        With check_crt, the full CRT value over all L primes is also formed
        and must agree (it does whenever |m| < q_0 / 2)."""
        q0 = self.q[0]
        m0 = (ct.c[0, 0] + self.mul(ct.c[1, 0], self.s[0], 0)) % np.uint64(q0)
        out = np.array([int(v) - q0 if int(v) > (q0 - 1) // 2 else int(v) for v in m0],
                       dtype=np.int64)
        if check_crt and ct.level > 1:
            Q = 1
            for r in range(ct.level):
                Q *= self.q[r]
            full = [0] * self.N
            for r in range(ct.level):
                q = self.q[r]
                mr = (ct.c[0, r] + self.mul(ct.c[1, r], self.s[r], r)) % np.uint64(q)
                Qr = Q // q
                coef = Qr * pow(Qr, -1, q)
                for k in range(self.N):
                    full[k] += int(mr[k]) * coef
            for k in range(self.N):
                v = full[k] % Q
                if v > (Q - 1) // 2:
                    v -= Q
                assert v == int(out[k]), "CRT reconstruction disagrees with q0 lift"
        return out

    # -- homomorphic operations -------------------------------------------
    def add(self, a, b):
        """Sum of two ciphertexts at one level whose nominal scales agree to a
        relative 2^-40; the result keeps a's nominal scale."""
        assert a.level == b.level, "level mismatch"
        assert abs(a.scale - b.scale) <= abs(a.scale) * 2.0 ** -40, "scale mismatch"
        c = np.empty_like(a.c)
        for r in range(a.level):
            c[:, r] = (a.c[:, r] + b.c[:, r]) % np.uint64(self.q[r])
        return Ciphertext(c, a.level, a.scale)

    def mul_const(self, a, C, sigma):
        """ct * C for an integer constant C = llround(value * sigma)."""
        c = np.empty_like(a.c)
        for r in range(a.level):
            q = self.q[r]
            for k in range(a.c.shape[0]):
                c[k, r] = core.vec_mul_scalar(a.c[k, r], C % q, q)
        return Ciphertext(c, a.level, a.scale * sigma)

    def add_const(self, a, C):
        """ct + C for an integer constant polynomial (C, 0, ..., 0)."""
        c = a.c.copy()
        for r in range(a.level):
            q = self.q[r]
            c[0, r, 0] = (int(c[0, r, 0]) + C % q) % q
        return Ciphertext(c, a.level, a.scale)

    def tensor(self, a, b):
        """(a0 b0, a0 b1 + a1 b0, a1 b1)"""
        assert a.level == b.level
        L = a.level
        d = np.zeros((3, L, self.N), dtype=np.uint64)
        for r in range(L):
            q = np.uint64(self.q[r])
            d[0, r] = self.mul(a.c[0, r], b.c[0, r], r)
            d[1, r] = (self.mul(a.c[0, r], b.c[1, r], r) + self.mul(a.c[1, r], b.c[0, r], r)) % q
            d[2, r] = self.mul(a.c[1, r], b.c[1, r], r)
        return Ciphertext(d, L, a.scale * b.scale)

    def keyswitch_accumulate(self, d2, L, key=None):
        """Inner product of the per-prime digits with the key: digit j is
        residue j of d2 ([L][N], coefficient form) lifted to [0, q_j) and
        reduced into every prime of q_0..q_{L-1}, P;
        acc_k = sum_j digit_j * ksk_j[k]  over those L+1 primes
        (key: the relinearisation key unless another is given)."""
        N, Lt = self.N, self.L_top
        ksk = self.ksk if key is None else key
        targets = list(range(L)) + [Lt]          # key residue indices
        acc = np.zeros((2, L + 1, N), dtype=np.uint64)
        for j in range(L):
            D = d2[j]
            for ti, kr in enumerate(targets):
                p = self.key_primes[kr]
                Dt = D % np.uint64(p)
                for k in range(2):
                    prod = self.mul(Dt, ksk[j, k, kr], kr)
                    acc[k, ti] = (acc[k, ti] + prod) % np.uint64(p)
        return acc

    def mod_down(self, acc, L):
        """ModDown by P: out_t = (acc_t - [v]_{q_t}) * P^{-1} mod q_t, v the
        centred residue of acc mod P (P odd: no ties)."""
        out = np.zeros((acc.shape[0], L, self.N), dtype=np.uint64)
        for k in range(acc.shape[0]):
            for t in range(L):
                q = self.q[t]
                v = centred_mod(acc[k, L], self.P, q)
                diff = (acc[k, t] + np.uint64(q) - v) % np.uint64(q)
                out[k, t] = core.vec_mul_scalar(diff, pow(self.P, -1, q), q)
        return out

    def keyswitch(self, d2, L):
        """RNS key switching with per-prime digits and one special prime."""
        return self.mod_down(self.keyswitch_accumulate(d2, L), L)

    def relinearise(self, d):
        ks = self.keyswitch(d.c[2], d.level)
        c = np.empty((2, d.level, self.N), dtype=np.uint64)
        for r in range(d.level):
            q = np.uint64(self.q[r])
            c[0, r] = (d.c[0, r] + ks[0, r]) % q
            c[1, r] = (d.c[1, r] + ks[1, r]) % q
        return Ciphertext(c, d.level, d.scale)

    def rescale(self, a):
        """Divide by the last prime q_{L-1} with the centred remainder:
        out_i = (c_i - [v]_{q_i}) q_{L-1}^{-1} mod q_i, i < L-1."""
        L = a.level
        assert L >= 2, "no prime left to rescale by"
        ql = self.q[L - 1]
        k_comp = a.c.shape[0]
        c = np.zeros((k_comp, L - 1, self.N), dtype=np.uint64)
        for k in range(k_comp):
            for i in range(L - 1):
                q = self.q[i]
                v = centred_mod(a.c[k, L - 1], ql, q)
                diff = (a.c[k, i] + np.uint64(q) - v) % np.uint64(q)
                c[k, i] = core.vec_mul_scalar(diff, pow(ql, -1, q), q)
        return Ciphertext(c, L - 1, a.scale / float(ql))

    def mod_drop(self, a, to_level):
        """Delete residues above to_level (no scaling)."""
        return Ciphertext(a.c[:, :to_level].copy(), to_level, a.scale)

    # -- network blocks (the scale schedule) ------------------------------
    def linear(self, xs, rows, bias):
        """Dense / convolution block (Eq. cnn with the bias added once after
        the sum): y_o = rescale(sum_i llround(w_oi * q_{L-1}) x_i) + llround(b_o * s_y).
        rows: list of (input indices, weights) per output."""
        L = xs[0].level
        s = xs[0].scale
        qd = float(self.q[L - 1])
        out = []
        for o, (idx, ws) in enumerate(rows):
            acc = np.zeros((2, L, self.N), dtype=np.uint64)
            for i, w in zip(idx, ws):
                x = xs[i]
                assert x.level == L and x.scale == s
                W = llround(float(w) * qd)
                for r in range(L):
                    q = self.q[r]
                    for k in range(2):
                        core.vec_mac_scalar(acc[k, r], x.c[k, r], W % q, q)
            y = self.rescale(Ciphertext(acc, L, s * qd))
            y = self.add_const(y, llround(float(bias[o]) * y.scale))
            out.append(y)
        return out

    def square(self, x):
        """x^2 = rescale(relinearise(x (x) x)), one level."""
        return self.rescale(self.relinearise(self.tensor(x, x)))

    def affine(self, x, a):
        """a0 + a1 x in one level, like a one-term linear block:
            y = rescale(x * llround(a1 * q)) + llround(a0 * scale(y)),  q = q_{L-1}"""
        L = x.level
        assert L >= 2, "an affine activation needs one level"
        q = float(self.q[L - 1])
        y = self.rescale(self.mul_const(x, llround(float(a[1]) * q), q))
        return self.add_const(y, llround(float(a[0]) * y.scale))

    def poly2(self, x, a):
        """a0 + a1 x + a2 x^2 in two levels (Eq. relu_approximate has this
        form); the degree-3 schedule without its cubic term:
            x2 = rescale(relin(x (x) x))                     scale s2 = s*s/q
            T  = x2 * llround(a2 * s_2) + drop(x) * llround(a1 * q'),  s_2 = s*q'/s2
            y  = rescale(T) + llround(a0 * scale(y))"""
        L = x.level
        assert L >= 3, "a degree-2 activation needs two levels"
        q = float(self.q[L - 1])
        qp = float(self.q[L - 2])
        s = x.scale
        s2 = (s * s) / q
        x2 = self.rescale(self.relinearise(self.tensor(x, x)))
        sg2 = (s * qp) / s2
        t2 = self.mul_const(x2, llround(float(a[2]) * sg2), sg2)
        t3 = self.mul_const(self.mod_drop(x, L - 1), llround(float(a[1]) * qp), qp)
        y = self.rescale(self.add(t2, t3))
        return self.add_const(y, llround(float(a[0]) * y.scale))

    def poly(self, x, a):
        """Polynomial activation of degree len(a) - 1 (1 .. 31)."""
        d = len(a) - 1
        if d == 1:
            return self.affine(x, a)
        if d == 2:
            return self.poly2(x, a)
        if d == 3:
            return self.poly3(x, a)
        if 4 <= d <= MAX_POLY_DEGREE:
            return self.poly_powers(x, a)
        raise ValueError("polynomial degree %d (1..%d supported)" % (d, MAX_POLY_DEGREE))

    def poly_powers(self, x, a):
        """Degree d >= 4 in ceil(log2 d) + 1 levels.  Powers: x^(2^j) by
        squaring, any other x^i = x^(2^j) x^(i - 2^j) (2^j the largest power of
        two below i), each product relinearised and rescaled, the operand at
        the higher level first mod-dropped to the other's level.  With l* the
        lowest level among the powers and S = s q_{l*-1} (s the scale of x):
            T = sum_{i >= 1, a_i != 0} drop(x^i, l*) * llround(a_i * S / s_i)
            y = rescale(T) + llround(a0 * scale(y))
        (s_i the scale of x^i; the terms are added in increasing i)."""
        d = len(a) - 1
        pw = {1: x}
        for i in range(2, d + 1):
            j = 1 << (i.bit_length() - 1)
            if j == i:
                j = i // 2
            A, B = pw[j], pw[i - j]
            lv = min(A.level, B.level)
            assert lv >= 2, "not enough levels for degree %d" % d
            A = A if A.level == lv else self.mod_drop(A, lv)
            B = B if B.level == lv else self.mod_drop(B, lv)
            pw[i] = self.rescale(self.relinearise(self.tensor(A, B)))
        lstar = min(p.level for p in pw.values())
        assert lstar >= 2, "not enough levels for degree %d" % d
        S = x.scale * float(self.q[lstar - 1])
        T = None
        for i in range(1, d + 1):
            if float(a[i]) == 0.0:
                continue
            p = pw[i] if pw[i].level == lstar else self.mod_drop(pw[i], lstar)
            sig = S / p.scale
            t = self.mul_const(p, llround(float(a[i]) * sig), sig)
            T = t if T is None else self.add(T, t)
        assert T is not None, "polynomial without non-constant terms"
        y = self.rescale(T)
        return self.add_const(y, llround(float(a[0]) * y.scale))

    def poly3(self, x, a):
        """a0 + a1 x + a2 x^2 + a3 x^3 in two levels (Eq. sigmoid_approximate
        has this form).  With q = q_{L-1}, q' = q_{L-2} and s the scale of x:
            x2 = rescale(relin(x (x) x))                     scale s2 = s*s/q
            w  = rescale(x * llround(a3 * s3)),  s3 = q'*q/s2
            T  = relin(x2 (x) w) + x2 * llround(a2 * s_2) + drop(x) * llround(a1 * q'),
                 s_2 = s*q'/s2
            y  = rescale(T) + llround(a0 * scale(y))"""
        L = x.level
        assert L >= 3, "a degree-3 activation needs two levels"
        q = float(self.q[L - 1])
        qp = float(self.q[L - 2])
        s = x.scale
        s2 = (s * s) / q
        x2 = self.rescale(self.relinearise(self.tensor(x, x)))
        s3 = (qp * q) / s2
        w = self.rescale(self.mul_const(x, llround(float(a[3]) * s3), s3))
        t1 = self.relinearise(self.tensor(x2, w))
        sg2 = (s * qp) / s2
        t2 = self.mul_const(x2, llround(float(a[2]) * sg2), sg2)
        t3 = self.mul_const(self.mod_drop(x, L - 1), llround(float(a[1]) * qp), qp)
        T = self.add(self.add(t1, t2), t3)
        y = self.rescale(T)
        return self.add_const(y, llround(float(a[0]) * y.scale))


# ---------------------------------------------------------------------------
# Graph evaluation: Alg. firing / signal_carrier / get_inbound_signal /
# apply_signal / set_outbound_signals (Sec. 3, graph rules list).
# ---------------------------------------------------------------------------
def _in_edges(graph, n):
    return [e for e, (a, b) in enumerate(graph["edges"]) if b == n]


def _out_edges(graph, n):
    return [e for e, (a, b) in enumerate(graph["edges"]) if a == n]


def fire(graph, inputs, signals, apply_fn, match_fn):
    """Alg. firing: carry each input signal through the graph in turn.
    apply_fn(node_index, node, stacked_input) -> output list (or None).
    Returns {output node index: signal}.  A node fires only once every
    in-edge carries a signal; its output is broadcast to every out-edge;
    after setting its outputs it carries on into its successors."""
    edge_sig = {}
    outputs = {}
    fired = set()

    def get_inbound(n, bootstrap):
        if bootstrap is not None:
            return bootstrap
        ins = _in_edges(graph, n)
        if any(e not in edge_sig for e in ins):
            return None
        s = [edge_sig[e] for e in ins]
        if len(s) == 1:
            return s[0]
        return match_fn(s)

    def carrier(n, bootstrap):
        if n in fired:
            return
        s = get_inbound(n, bootstrap)
        if s is None:
            return
        s = apply_fn(n, graph["nodes"][n], s)
        if s is None:
            return
        fired.add(n)
        if graph["nodes"][n]["kind"] == "output":
            outputs[n] = s
        for e in _out_edges(graph, n):
            edge_sig[e] = s
        seen = []
        for e in _out_edges(graph, n):
            b = graph["edges"][e][1]
            if b not in seen:
                seen.append(b)
                carrier(b, None)

    for i, n in enumerate(inputs):
        carrier(n, signals[i])
    return outputs


def _stack_cts(ctx, sigs, kind):
    """Stack per-edge signals (edge order).  'add' nodes sum them element by
    element; other nodes concatenate.  Levels are matched by mod-drop."""
    Lmin = min(ct.level for sig in sigs for ct in sig)
    sigs = [[ct if ct.level == Lmin else ctx.mod_drop(ct, Lmin) for ct in sig] for sig in sigs]
    return {"edges": sigs}


def eval_graph(ctx, graph, inputs, signals):
    """Encrypted evaluation of the graph over lists of ciphertexts."""

    def apply_fn(n, node, s):
        if isinstance(s, dict):
            edges = s["edges"]
            if node["kind"] == "add":
                out = edges[0]
                for sig in edges[1:]:
                    out = [ctx.add(a, b) for a, b in zip(out, sig)]
                return out
            s = [ct for sig in edges for ct in sig]
        k = node["kind"]
        if k in ("input", "output"):
            return s
        if k == "linear":
            return ctx.linear(s, csr_rows(node), node["bias"])
        if k == "conv_packed":
            return ctx.conv_packed(s, node)
        if k == "poly":
            return [ctx.poly(x, node["coeffs"]) for x in s]
        if k == "relu":
            a = relu_coeffs(node["q"])
            return [ctx.poly(x, a) for x in s]
        if k == "square":
            return [ctx.square(x) for x in s]
        if k == "add":
            return s
        raise ValueError(k)

    return fire(graph, inputs, signals, apply_fn, lambda sigs: _stack_cts(ctx, sigs, None))


def packed_valid_slots(node, M):
    """Output slots b S + s r W + s c of a packed convolution (b < images,
    r, c < output side), in image, row, column order."""
    S, W, st, k = node["slot_stride"], node["W"], node["stride"], node["k"]
    OH = (node["H"] - k) // st + 1
    OW = (W - k) // st + 1
    idx = [b * S + st * r * W + st * c for b in range(node["images"]) for r in range(OH) for c in range(OW)]
    assert max(idx) < M
    return np.array(idx, dtype=np.int64)


def relayout_packed(z, node, n_in):
    """Client side of a refresh after a packed convolution: decoded filter
    ciphertexts z [F * n_in][slots] (filter-major) -> one row per feature
    f * OH * OW + r * OW + c, one column per image i * images + b."""
    F = node["filters"]
    M = z.shape[1]
    valid = packed_valid_slots(node, M)
    per_img = len(valid) // node["images"]
    out = np.zeros((F * per_img, M))
    for f in range(F):
        for i in range(n_in):
            v = z[f * n_in + i][valid].reshape(node["images"], per_img)
            for b in range(node["images"]):
                out[f * per_img:(f + 1) * per_img, i * node["images"] + b] = v[b]
    return out


def refresh_ct_id(node, k):
    """Object id of the k-th ciphertext re-encrypted at rotation node `node`."""
    return (1 << 40) + (node << 20) + k


def eval_graph_grouped(ctxs, graph, signals):
    """Encrypted evaluation of a graph with rotation (client refresh) nodes.
    Alg. autoHE over the input and rotation nodes gives the parameter groups;
    ctxs maps group id -> Context (its parameter set, keys generated).
    signals: per input node (node order), its list of ciphertexts encrypted
    under its group's context.  Every node computes in the context of the
    group it belongs to; a rotation node hands its ciphertexts to the client,
    which decrypts and decodes them under the upstream group's keys and
    encodes and encrypts them under the rotation's own group
    (ct id refresh_ct_id(node, k)).  Returns {output node: [Ciphertext]}."""
    from .params import autohe, ingress_nodes
    ing = ingress_nodes(graph)
    group_of, _, sources = autohe(graph, ing)

    def group_above(n):
        gs = {group_of[k] for k in sources.get(n, {})}
        assert len(gs) == 1, "node %d is reached from several parameter groups" % n
        return gs.pop()

    def apply_fn(n, node, s):
        if isinstance(s, dict):
            edges = s["edges"]
            if node["kind"] == "add":
                ctx = ctxs[group_above(n)]
                out = edges[0]
                for sig in edges[1:]:
                    out = [ctx.add(a, b) for a, b in zip(out, sig)]
                return out
            s = [ct for sig in edges for ct in sig]
        k = node["kind"]
        if k in ("input", "output"):
            return s
        if k == "rotate":
            up, down = ctxs[group_above(n)], ctxs[group_of[n]]
            z = np.stack([up.decode(up.decrypt(ct), ct.scale) for ct in s])
            if "relayout" in node:                    # client re-packs the slots
                geo = node["relayout"]
                z = relayout_packed(z, geo, len(s) // geo["filters"])
            Md = down.N // 2
            if z.shape[1] < Md:
                z = np.pad(z, ((0, 0), (0, Md - z.shape[1])))
            return [down.encrypt(down.encode(z[i]), refresh_ct_id(n, i)) for i in range(z.shape[0])]
        ctx = ctxs[group_above(n)]
        if k == "conv_packed":
            return ctx.conv_packed(s, node)
        if k == "linear":
            return ctx.linear(s, csr_rows(node), node["bias"])
        if k == "poly":
            return [ctx.poly(x, node["coeffs"]) for x in s]
        if k == "relu":
            return [ctx.poly(x, relu_coeffs(node["q"])) for x in s]
        if k == "square":
            return [ctx.square(x) for x in s]
        raise ValueError(k)

    some = next(iter(ctxs.values()))
    inputs = [i for i in ing if graph["nodes"][i]["kind"] == "input"]
    return fire(graph, inputs, signals, apply_fn, lambda sigs: _stack_cts(some, sigs, None))


def relu_coeffs(q):
    """Eq. relu_approximate: R(x) ~ 4/(3 pi q) x^2 + x/2 + q/(3 pi) on [-q, q]
    (q: the approximation range), as [a0, a1, a2] in FP64."""
    q = float(q)
    return [q / (3 * math.pi), 0.5, 4 / (3 * math.pi * q)]


def csr_rows(node):
    rp, ci, w = node["row_ptr"], node["col_idx"], node["weight"]
    return [(ci[rp[o]:rp[o + 1]], w[rp[o]:rp[o + 1]]) for o in range(len(rp) - 1)]


def forward_fp64(graph, inputs, signals):
    """FP64 plaintext forward pass with the same polynomial activations.
    signals: per input node, a float64 array [n_ct][slots]."""

    def apply_fn(n, node, s):
        if isinstance(s, dict):
            edges = s["edges"]
            if node["kind"] == "add":
                out = edges[0]
                for sig in edges[1:]:
                    out = out + sig
                return out
            s = np.concatenate(edges, axis=0)
        k = node["kind"]
        if k in ("input", "output"):
            return s
        if k == "rotate":
            return relayout_packed(s, node["relayout"], s.shape[0] // node["relayout"]["filters"]) \
                if "relayout" in node else s
        if k == "conv_packed":
            F, kk = node["filters"], node["k"]
            valid = packed_valid_slots(node, s.shape[1])
            W_ = np.asarray(node["weight"], dtype=np.float64).reshape(F, kk * kk)
            offs = [dr * node["W"] + dc for dr in range(kk) for dc in range(kk)]
            out = np.zeros((F * s.shape[0], s.shape[1]))
            for f in range(F):
                for i in range(s.shape[0]):
                    acc = np.zeros(s.shape[1])
                    for p, o in enumerate(offs):
                        acc[valid] += W_[f, p] * np.roll(s[i], -o)[valid]
                    acc[valid] += float(node["bias"][f])
                    out[f * s.shape[0] + i] = acc
            return out
        if k == "linear":
            rows = csr_rows(node)
            out = np.zeros((len(rows), s.shape[1]))
            for o, (idx, ws) in enumerate(rows):
                for i, w in zip(idx, ws):
                    out[o] += float(w) * s[i]
                out[o] += float(node["bias"][o])
            return out
        if k in ("poly", "relu"):
            a = node["coeffs"] if k == "poly" else relu_coeffs(node["q"])
            out = np.zeros_like(s) + a[0]
            p = np.ones_like(s)
            for ak in a[1:]:
                p = p * s
                out = out + ak * p
            return out
        if k == "square":
            return s * s
        raise ValueError(k)

    return fire(graph, inputs, signals, apply_fn, lambda sigs: {"edges": sigs})


def graph_depth(graph, inputs):
    """Largest group cost (Alg. autoHE) -- convenience for tests."""
    from .params import autohe
    return max(autohe(graph, inputs)[1])
