"""BFV with RNS limbs (symmetric and public-key encryption) (oracle; test infrastructure only).

Sec. 2.2: BFV {N, t, q}; plaintexts in Z_t[X]/(X^N+1), ciphertexts in
(Z_q[X]/(X^N+1))^2; one plaintext-ciphertext product per linear layer, no
bootstrapping (Sec. 3.2.1).  Sec. 5: q is split into RNS limbs q_i < 2^64 and
all ring arithmetic is done per limb in the NTT domain.

Ciphertexts are kept in NTT form, limb-major: c[comp][limb][slot].

* keygen   : s ternary (from `sampling.ternary_secret`), stored as NTT(s) per limb.
* encrypt  : c1 = a (uniform, drawn directly in the NTT domain),
             c0 = NTT([q m / t] + e) - a * NTT(s), [.] rounding to nearest
             (= Delta m + [(q mod t) m / t], the scaling of SEAL, which the
             paper's GPU BFV follows): a plaintext-ciphertext product then
             carries no (q mod t) x overflow term, so products of two uniform
             Z_t values decrypt correctly at t = 2^59, q ~ 2^180 (Sec. 6).
* pk_keygen: public key (Sec. 2.2's BFV [Fan-Vercauteren]; the paper's
             simulators exchange pk): p1 = a uniform (NTT form),
             p0 = -(a * NTT(s)) - NTT(e).
* encrypt_pk: u ternary, e1, e2 errors;  c0 = NTT([q m / t] + e1) + NTT(u) * p0,
             c1 = NTT(e2) + NTT(u) * p1, so c0 + c1 s = [q m / t] + e1 - u e + e2 s.
* add_plain: c0 += NTT([q m' / t])   (Alg. 1 step 2: adding the MO's share).
* encode   : a signed integer polynomial lifted to every limb, in NTT form.
* decrypt  : x = INTT(c0 + c1 * NTT(s)) per limb, recombined exactly by the
             Chinese remainder theorem into [0, q), and
             m = round(t * x / q) mod t = floor((2 t x + q) / (2 q)) mod t.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Sequence

import numpy as np

from .ntt import intt_radix2, ntt_radix2
from .params import BfvParams
from .philox import DOMAIN_PK_A, DOMAIN_PK_E, DOMAIN_PK_E2
from .sampling import gaussian_error, ternary_secret, ternary_u, uniform_a


@dataclass
class SecretKey:
    s: List[int]                 # ternary coefficients
    s_hat: np.ndarray            # object array [L][N], NTT(s mod q_i)


def keygen(p: BfvParams, seed: int) -> SecretKey:
    s = ternary_secret(seed, p.n)
    s_hat = np.stack([ntt_radix2([x % q for x in s], q, psi)
                      for q, psi in zip(p.primes, p.psis)])
    return SecretKey(s=s, s_hat=s_hat)


def lift_plain(p: BfvParams, values: Sequence[int]) -> np.ndarray:
    """Signed integer polynomial -> object array [L][N] of residues (coefficient form)."""
    return np.stack([np.array([int(v) % q for v in values], dtype=object) for q in p.primes])


def to_ntt(p: BfvParams, coeffs: np.ndarray) -> np.ndarray:
    return np.stack([ntt_radix2(coeffs[i], q, psi)
                     for i, (q, psi) in enumerate(zip(p.primes, p.psis))])


def from_ntt(p: BfvParams, slots: np.ndarray) -> np.ndarray:
    return np.stack([intt_radix2(slots[i], q, psi)
                     for i, (q, psi) in enumerate(zip(p.primes, p.psis))])


def centered(v: int, t: int) -> int:
    """Z_t value -> signed representative in [-t/2, t/2)."""
    v %= t
    return v - t if v >= t // 2 else v


def encode_plain(p: BfvParams, values: Sequence[int]) -> np.ndarray:
    """Plaintext multiplier: Z_t values lifted through their centred
    representative to every limb, NTT form [L][N]."""
    return to_ntt(p, lift_plain(p, [centered(int(v), p.t) for v in values]))


def scaled_message(p: BfvParams, m: Sequence[int], e: Sequence[int] | None = None) -> np.ndarray:
    """round(q m / t) + e per limb (m read in [0, t)), coefficient form."""
    Q, t = p.q, p.t
    if e is None:
        e = [0] * p.n
    sm = [(Q * (int(mi) % t) + t // 2) // t + int(ei) for mi, ei in zip(m, e)]
    return np.stack([np.array([v % q for v in sm], dtype=object) for q in p.primes])


def encrypt(p: BfvParams, sk: SecretKey, m: Sequence[int], seed: int, ct_index: int) -> np.ndarray:
    """Returns c[2][L][N] (NTT form).  Randomness: a from stream (seed, A, ct_index, limb),
    e from stream (seed, E, ct_index)."""
    e = gaussian_error(seed, ct_index, p.n, p.sigma)
    base = to_ntt(p, scaled_message(p, m, e))
    c0, c1 = [], []
    for i, q in enumerate(p.primes):
        a = np.array(uniform_a(seed, ct_index, i, p.n, q), dtype=object)
        c1.append(a)
        c0.append((base[i] - a * sk.s_hat[i]) % q)
    return np.stack([np.stack(c0), np.stack(c1)])


@dataclass
class PublicKey:
    p0: np.ndarray               # object array [L][N], NTT form
    p1: np.ndarray               # object array [L][N], NTT form (= a)


def pk_keygen(p: BfvParams, sk: SecretKey, seed: int) -> PublicKey:
    """pk = (-(a s + e), a) with a from stream (seed, PK_A, 0, limb), e from (seed, PK_E, 0)."""
    e_hat = to_ntt(p, lift_plain(p, gaussian_error(seed, 0, p.n, p.sigma, DOMAIN_PK_E)))
    p0, p1 = [], []
    for i, q in enumerate(p.primes):
        a = np.array(uniform_a(seed, 0, i, p.n, q, DOMAIN_PK_A), dtype=object)
        p1.append(a)
        p0.append((-(a * sk.s_hat[i]) - e_hat[i]) % q)
    return PublicKey(p0=np.stack(p0), p1=np.stack(p1))


def encrypt_pk(p: BfvParams, pk: PublicKey, m: Sequence[int], seed: int, ct_index: int) -> np.ndarray:
    """Public-key encryption, c[2][L][N] (NTT form).  Randomness of ciphertext
    ct_index: u from stream (seed, PK_U, ct_index), e1 from (seed, E, ct_index)
    (the symmetric encryption's error stream), e2 from (seed, PK_E2, ct_index)."""
    u_hat = to_ntt(p, lift_plain(p, ternary_u(seed, ct_index, p.n)))
    base0 = to_ntt(p, scaled_message(p, m, gaussian_error(seed, ct_index, p.n, p.sigma)))
    base1 = to_ntt(p, lift_plain(p, gaussian_error(seed, ct_index, p.n, p.sigma, DOMAIN_PK_E2)))
    c0, c1 = [], []
    for i, q in enumerate(p.primes):
        c0.append((base0[i] + u_hat[i] * pk.p0[i]) % q)
        c1.append((base1[i] + u_hat[i] * pk.p1[i]) % q)
    return np.stack([np.stack(c0), np.stack(c1)])


def add_plain(p: BfvParams, ct: np.ndarray, m: Sequence[int]) -> np.ndarray:
    """ct + round(q m / t) (Alg. 1 step 2, adding a plaintext share)."""
    out = ct.copy()
    add = to_ntt(p, scaled_message(p, m))
    for i, q in enumerate(p.primes):
        out[0, i] = (out[0, i] + add[i]) % q
    return out


def add_noise(p: BfvParams, ct: np.ndarray, f: Sequence[int]) -> np.ndarray:
    """c0 += NTT(f) for an integer polynomial f (flooding the noise of a returned
    ciphertext; its plaintext is unchanged while |noise + f| < Delta / 2)."""
    out = ct.copy()
    add = to_ntt(p, lift_plain(p, f))
    for i, q in enumerate(p.primes):
        out[0, i] = (out[0, i] + add[i]) % q
    return out


def sub_plain(p: BfvParams, ct: np.ndarray, m: Sequence[int]) -> np.ndarray:
    """ct - round(q m / t) (Alg. 1 step 3, subtracting the mask)."""
    out = ct.copy()
    sub = to_ntt(p, scaled_message(p, m))
    for i, q in enumerate(p.primes):
        out[0, i] = (out[0, i] - sub[i]) % q
    return out


def mul_plain(p: BfvParams, ct: np.ndarray, pt: np.ndarray) -> np.ndarray:
    """Ciphertext x plaintext product, element-wise in the NTT domain."""
    out = ct.copy()
    for i, q in enumerate(p.primes):
        out[0, i] = ct[0, i] * pt[i] % q
        out[1, i] = ct[1, i] * pt[i] % q
    return out


def add_ct(p: BfvParams, a: np.ndarray, b: np.ndarray) -> np.ndarray:
    out = a.copy()
    for i, q in enumerate(p.primes):
        out[:, i] = (a[:, i] + b[:, i]) % q
    return out


def crt(p: BfvParams, residues: Sequence[int]) -> int:
    q = p.q
    x = 0
    for r, qi in zip(residues, p.primes):
        qi_star = q // qi
        x += int(r) * qi_star * pow(qi_star, -1, qi)
    return x % q


def decrypt_phase(p: BfvParams, sk: SecretKey, ct: np.ndarray) -> List[int]:
    """x = c0 + c1 * s in [0, q), coefficient form (exact big integers)."""
    slots = np.stack([(ct[0, i] + ct[1, i] * sk.s_hat[i]) % q for i, q in enumerate(p.primes)])
    coeff = from_ntt(p, slots)
    return [crt(p, coeff[:, j]) for j in range(p.n)]


def decrypt(p: BfvParams, sk: SecretKey, ct: np.ndarray) -> List[int]:
    q, t = p.q, p.t
    return [((2 * t * x + q) // (2 * q)) % t for x in decrypt_phase(p, sk, ct)]


def noise_budget_ok(p: BfvParams, sk: SecretKey, ct: np.ndarray) -> bool:
    """True when every coefficient's t*x/q lies within 1/4 of an integer."""
    q, t = p.q, p.t
    for x in decrypt_phase(p, sk, ct):
        r = (t * x) % q
        if min(r, q - r) * 4 >= q:
            return False
    return True
