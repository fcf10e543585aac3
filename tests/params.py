"""Parameter sets used by the tests and the benchmark (plain data).

Prime chains: the smallest primes q = 1 (mod U) in [lo, hi).  U is a multiple
of 2N (negacyclic NTT) and of every plaintext modulus in use (q = 1 mod p).
"""
U50 = 2 ** 16 * 17 * 131 * 257          # 50-bit chain, N <= 2^15, p in {17, 131, 257}
U36 = 8192 * 17                          # 36-bit chain, N <= 2^12, p = 17
CHAIN50 = dict(U=U50, lo=2 ** 49, hi=2 ** 50)
CHAIN36 = dict(U=U36, lo=2 ** 35, hi=2 ** 36)

# name: (logN, p, d, L, K, chain)
SMALL_P17 = dict(logN=12, p=17, d=1, L=4, K=1, **CHAIN36)     # one LT, 4x36b + 1 special
MID_P131 = dict(logN=14, p=131, d=2, L=10, K=3, **CHAIN50)    # LT/EQ, 10x50b + 3 special
MAXMIN_P257 = dict(logN=15, p=257, d=2, L=20, K=4, **CHAIN50) # tournament, 20x50b + 4 special
