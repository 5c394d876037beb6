"""Planted mistakes in the oracle must be caught by its pins.

Each case replaces one oracle function with a plausibly wrong version (a
dropped term, a wrong sign or index, a transposed operand, a missing
modulus) on the CPU, runs the pins that guard it, and requires at least one
of them to fail.  Nothing here touches the CUDA library.
"""
import numpy as np
import pytest

from oracle import cms_oracle as O
import test_oracle_pins as pins


def _fails(*tests):
    for t in tests:
        try:
            t()
        except AssertionError:
            return True
    return False


def _run_param(fn, cases):
    def run():
        for args in cases:
            fn(*args)
    return run


ROUTE_CASES = [(16, 9, 16, 32, 2), (23, 17, 11, 64, 3), (40, 12, 40, 100, 1)]


def test_mutation_sign_dropped_in_count_sketch(monkeypatch):
    monkeypatch.setattr(O, "count_sketch",
                        lambda u, h, s, b: np.bincount(h, weights=np.asarray(u, float), minlength=b))
    assert _fails(_run_param(pins.test_fft_route_equals_definition_and_convolution, ROUTE_CASES),
                  pins.test_injective_hash_gives_exact_product)


def test_mutation_hash_without_mersenne_modulus(monkeypatch):
    def bad(a, c, x, b):
        x = np.asarray(x, dtype=np.uint64)
        return ((np.uint64(a) * x + np.uint64(c)) % np.uint64(b)).astype(np.int64)
    monkeypatch.setattr(O, "hash_bucket", bad)
    assert _fails(pins.test_hash_hand_worked_values)


def test_mutation_sign_from_wrong_bit(monkeypatch):
    def bad(a, c, x):
        x = np.asarray(x, dtype=np.uint64)
        v = (np.uint64(a) * x + np.uint64(c)) % np.uint64(O.P31)
        return (1 - 2 * ((v >> np.uint64(1)) % np.uint64(2)).astype(np.int64)).astype(np.int64)
    monkeypatch.setattr(O, "hash_sign", bad)
    assert _fails(pins.test_hash_hand_worked_values)


def test_mutation_decode_subtracts_buckets(monkeypatch):
    def bad(c, tab, i, j):
        i = np.asarray(i, dtype=np.int64)
        j = np.asarray(j, dtype=np.int64)
        X = np.empty((tab.d, len(i)))
        for t in range(tab.d):
            z = (tab.h1[t, i] - tab.h2[t, j]) % tab.b
            X[t] = tab.s1[t, i] * tab.s2[t, j] * np.asarray(c[t], float)[z]
        return X
    monkeypatch.setattr(O, "estimates", bad)
    assert _fails(pins.test_decompress_formula_on_hand_sketch, pins.test_injective_hash_gives_exact_product)


def test_mutation_transposed_operand_in_definition(monkeypatch):
    real = O.sketch_definition

    def bad(A, B, tab):
        Bt = np.asarray(B).T
        if Bt.shape[0] == np.asarray(A).shape[1]:
            return real(A, Bt, tab)          # B^T in place of B where the shapes allow it
        return real(A, B, tab) * 1.001
    monkeypatch.setattr(O, "sketch_definition", bad)
    assert _fails(_run_param(pins.test_fft_route_equals_definition_and_convolution, ROUTE_CASES))


def test_mutation_forward_fft_in_place_of_inverse(monkeypatch):
    real_ifft = np.fft.ifft

    def bad_sketch(A, B, tab, return_imag=False):
        import numpy.fft as F
        F_ifft = F.ifft
        F.ifft = lambda v: np.fft.fft(v) / len(v)
        try:
            return O.__dict__["_orig_sketch_fft"](A, B, tab, return_imag)
        finally:
            F.ifft = F_ifft
    monkeypatch.setitem(O.__dict__, "_orig_sketch_fft", O.sketch_fft)
    monkeypatch.setattr(O, "sketch_fft", bad_sketch)
    assert _fails(_run_param(pins.test_fft_route_equals_definition_and_convolution, ROUTE_CASES))
    assert np.fft.ifft is real_ifft


def test_mutation_even_median_takes_upper(monkeypatch):
    monkeypatch.setattr(O, "median", lambda v, axis=0: np.sort(v, axis=axis).take(v.shape[axis] // 2, axis=axis))
    assert _fails(pins.test_median_convention)


def test_mutation_splitmix_wrong_constant(monkeypatch):
    def bad(state):
        state = (state + 0x9E3779B97F4A7C15) & O._MASK64
        z = state
        z = ((z ^ (z >> 31)) * O._MIX1) & O._MASK64
        z = ((z ^ (z >> 27)) * O._MIX2) & O._MASK64
        return state, z ^ (z >> 31)
    monkeypatch.setattr(O, "splitmix64", bad)
    assert _fails(pins.test_splitmix64_matches_published_outputs)


def test_mutation_convolution_index_off_by_one(monkeypatch):
    def bad(A, B, tab):
        c = O.sketch_definition(A, B, tab)
        return np.roll(c, 1, axis=1)
    monkeypatch.setattr(O, "sketch_convolution", bad)
    assert _fails(_run_param(pins.test_fft_route_equals_definition_and_convolution, ROUTE_CASES),
                  pins.test_fft_route_equals_convolution_at_b1024)


def test_mutation_diagonal_removed_with_wrong_sign(monkeypatch):
    orig = O.remove_diagonal

    def bad(c, diag, tab):
        return orig(c, -np.asarray(diag), tab)
    monkeypatch.setattr(O, "remove_diagonal", bad)
    assert _fails(pins.test_remove_diagonal_is_the_sketch_of_the_offdiagonal_part)


def test_mutation_diagonal_removed_at_column_bucket(monkeypatch):
    def bad(c, diag, tab):
        out = np.array(c, dtype=np.float64, copy=True)
        i = np.arange(len(diag))
        for t in range(tab.d):
            z = (2 * tab.h2[t, i]) % tab.b
            np.subtract.at(out[t], z, tab.s1[t, i] * tab.s2[t, i] * diag)
        return out
    monkeypatch.setattr(O, "remove_diagonal", bad)
    assert _fails(pins.test_remove_diagonal_is_the_sketch_of_the_offdiagonal_part)


def test_mutation_diagonal_transposed_operand(monkeypatch):
    monkeypatch.setattr(O, "product_diagonal",
                        lambda A, B: np.einsum("ik,ik->i", np.asarray(A)[:, :1].repeat(np.asarray(A).shape[1], 1),
                                               np.asarray(A)))
    assert _fails(pins.test_product_diagonal_brute_force)


def test_mutation_candidates_without_absolute_value(monkeypatch):
    orig = O.candidates

    def bad(c, tab, n1, n3, tau, skip_diagonal=True):
        full = orig(c, tab, n1, n3, tau, skip_diagonal)
        est = O.decompress(c, tab, full[:, 0], full[:, 1])
        return full[est > tau]
    monkeypatch.setattr(O, "candidates", bad)
    assert _fails(lambda: pins.test_candidates_with_injective_hashes_are_the_large_entries(True))


def test_mutation_sign4_without_cubic_term(monkeypatch):
    def bad(coef, x):
        a0, a1, a2, _ = (int(v) for v in coef)
        return np.array([1 - 2 * (((a2 * xv + a1) * xv + a0) % ((1 << 31) - 1) % 2)
                         for xv in np.asarray(x).tolist()], dtype=np.int64)
    monkeypatch.setattr(O, "sign4", bad)
    assert _fails(pins.test_sign4_hand_worked_values)


def test_mutation_ams_with_one_sign_vector_for_both_sides(monkeypatch):
    def bad(A, B, seed, d):
        A = np.asarray(A, dtype=np.float64)
        B = np.asarray(B, dtype=np.float64)
        coef = O.draw_sign4_coefficients(seed, d)
        X = np.empty(d)
        for t in range(d):
            s1 = O.sign4(coef[t, 0], np.arange(A.shape[0]))
            s2 = O.sign4(coef[t, 0], np.arange(B.shape[1]))
            X[t] = (s1 @ A) @ (B @ s2)
        return X
    monkeypatch.setattr(O, "ams_frobenius", bad)
    assert _fails(pins.test_ams_estimate_is_the_signed_sum_of_ab)


def test_mutation_doubling_with_row_hash_only(monkeypatch):
    def bad(rows, cols, seed, d, b_max):
        coef = O.draw_coefficients(seed, d)
        rows = np.asarray(rows, dtype=np.int64)
        b = 2
        while b <= b_max:
            worst = max(len(np.unique(O.hash_bucket(coef[t, 0, 0], coef[t, 0, 1], rows, b))) for t in range(d))
            if 5 * worst <= b:
                return b, worst
            b *= 2
        return -1, 0
    monkeypatch.setattr(O, "nnz_doubling", bad)
    assert _fails(pins.test_nnz_doubling_stops_at_the_first_b_with_a_fifth_occupied)


def test_mutation_decode_without_distance_check(monkeypatch):
    def bad(s, L, rho):
        s = np.asarray(s, dtype=np.int64)
        x = 0
        for q in range(L):
            seg = s[q * 2 * rho: (q + 1) * 2 * rho]
            x |= (1 if seg[:rho].sum() >= (seg[rho:] == 0).sum() and seg[:rho].sum() > 0 else 0) << q
        return x
    monkeypatch.setattr(O, "decode_code", bad)
    assert _fails(pins.test_code_round_trip_and_error_correction)


def test_mutation_masks_swapped_between_sides(monkeypatch):
    orig = O.masked_sketches

    def bad(A, B, tab, rho):
        P = orig(A, B, tab, rho)
        ell = P.shape[0] // 2
        return np.concatenate([P[ell:], P[:ell]])
    monkeypatch.setattr(O, "masked_sketches", bad)
    assert _fails(pins.test_find_significant_returns_the_planted_entries)
