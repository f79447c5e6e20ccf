// Host-side construction of GF(p^k) and of the tables the kernels read.
//
// Sec. 7: the field is Z_p[X]/(P) with P irreducible of degree k; elements
// are stored as discrete logarithms of a generator and converted with
// tables.  Sec. 2 / Thm. 1 (Eq. 2) fix the q-adic radix and block size,
// Eq. 3 the plane-accumulation bound, Thm. 3 the two correction-and-fold
// tables that replace the radix conversion and the division by P.
#include <cstring>

#include "qadic_internal.h"

namespace qadic {

namespace {

using Poly = std::vector<int64_t>;   // coefficients low -> high, in [0, p-1]

void trim(Poly &a) {
    while (!a.empty() && a.back() == 0) a.pop_back();
}

int64_t inv_mod(int64_t a, int64_t p) {   // Fermat, p prime
    int64_t r = 1, b = ((a % p) + p) % p, e = p - 2;
    while (e > 0) {
        if (e & 1) r = r * b % p;
        b = b * b % p;
        e >>= 1;
    }
    return r;
}

// a mod m (m need not be monic), over Z_p.
Poly pmod(Poly a, const Poly &m, int64_t p) {
    trim(a);
    const int64_t lead_inv = inv_mod(m.back(), p);
    const size_t dm = m.size() - 1;
    while (a.size() > dm) {
        const int64_t c = a.back() * lead_inv % p;
        const size_t shift = a.size() - 1 - dm;
        for (size_t i = 0; i <= dm; ++i)
            a[shift + i] = ((a[shift + i] - c * m[i]) % p + p) % p;
        trim(a);
    }
    return a;
}

Poly pmulmod(const Poly &a, const Poly &b, const Poly &m, int64_t p) {
    if (a.empty() || b.empty()) return {};
    Poly r(a.size() + b.size() - 1, 0);
    for (size_t i = 0; i < a.size(); ++i)
        for (size_t j = 0; j < b.size(); ++j) r[i + j] = (r[i + j] + a[i] * b[j]) % p;
    return pmod(r, m, p);
}

Poly ppowmod(Poly base, uint64_t e, const Poly &m, int64_t p) {
    Poly r{1};
    base = pmod(base, m, p);
    while (e > 0) {
        if (e & 1) r = pmulmod(r, base, m, p);
        base = pmulmod(base, base, m, p);
        e >>= 1;
    }
    return r;
}

Poly pgcd(Poly a, Poly b, int64_t p) {
    trim(a);
    trim(b);
    while (!b.empty()) {
        Poly r = pmod(a, b, p);
        a = b;
        b = r;
    }
    return a;
}

uint64_t upow(uint64_t b, uint32_t e) {
    uint64_t r = 1;
    while (e--) r *= b;
    return r;
}

std::vector<uint64_t> prime_divisors(uint64_t n) {
    std::vector<uint64_t> out;
    for (uint64_t d = 2; d * d <= n; ++d) {
        if (n % d == 0) {
            out.push_back(d);
            while (n % d == 0) n /= d;
        }
    }
    if (n > 1) out.push_back(n);
    return out;
}

}  // namespace

bool is_prime(uint32_t p) {
    if (p < 2) return false;
    for (uint32_t d = 2; (uint64_t)d * d <= p; ++d)
        if (p % d == 0) return false;
    return true;
}

// Ben-Or's test: P of degree k is irreducible over Z_p iff
// gcd(X^(p^i) - X mod P, P) = 1 for every i = 1..floor(k/2).
bool poly_irreducible(uint32_t p, uint32_t k, const uint32_t *P) {
    if (k == 0 || P[k] != 1) return false;
    for (uint32_t i = 0; i <= k; ++i)
        if (P[i] >= p) return false;
    if (k == 1) return true;
    Poly m(P, P + k + 1);
    Poly xp{0, 1};   // X^(p^i) mod P, i = 0
    for (uint32_t i = 1; i <= k / 2; ++i) {
        xp = ppowmod(xp, p, m, p);
        Poly d = xp;
        d.resize(std::max<size_t>(d.size(), 2), 0);
        d[1] = ((d[1] - 1) % (int64_t)p + p) % p;
        trim(d);
        if (d.empty()) return false;           // X^(p^i) = X: a factor of degree | i
        Poly g = pgcd(m, d, p);
        if (g.size() > 1) return false;
    }
    return true;
}

int build_field(Field &f, uint32_t p, uint32_t k, const uint32_t *poly) {
    if (k < 1 || k > kMaxK) return set_error(QADIC_E_INVALID, "k=%u outside [1, %u]", k, kMaxK);
    if (p < 2 || p > 251) return set_error(QADIC_E_INVALID, "p=%u outside [2, 251]", p);
    if (!is_prime(p)) return set_error(QADIC_E_NOT_PRIME, "p=%u is not prime", p);
    const uint64_t order = upow(p, k);
    if (order > 65536)
        return set_error(QADIC_E_INVALID, "p^k=%llu exceeds 65536", (unsigned long long)order);
    f.p = p;
    f.k = k;
    f.order = (uint32_t)order;
    f.h = (p == 2) ? 1 : (p - 1) / 2;

    // Defining polynomial: given, or the smallest by sum a_i p^i (low coeffs).
    if (poly) {
        for (uint32_t i = 0; i <= k; ++i) f.poly[i] = poly[i];
        if (f.poly[k] != 1) return set_error(QADIC_E_INVALID, "defining polynomial must be monic");
        for (uint32_t i = 0; i <= k; ++i)
            if (f.poly[i] >= p) return set_error(QADIC_E_INVALID, "poly coefficient >= p");
        if (!poly_irreducible(p, k, f.poly))
            return set_error(QADIC_E_REDUCIBLE, "defining polynomial is reducible mod %u", p);
    } else {
        bool found = false;
        for (uint64_t v = 0; v < order && !found; ++v) {
            uint64_t t = v;
            for (uint32_t i = 0; i < k; ++i) {
                f.poly[i] = (uint32_t)(t % p);
                t /= p;
            }
            f.poly[k] = 1;
            found = poly_irreducible(p, k, f.poly);
        }
        if (!found) return set_error(QADIC_E_INVALID, "no irreducible polynomial found");
    }
    const Poly m(f.poly, f.poly + k + 1);

    // Generator: smallest element (by sum c_i p^i) whose powers g^(N/r) are
    // all != 1 for the primes r | N = p^k - 1 (Lagrange).
    const uint64_t N = order - 1;
    const std::vector<uint64_t> rs = prime_divisors(N);
    Poly g;
    for (uint64_t v = 1; v < order; ++v) {
        Poly a(k, 0);
        uint64_t t = v;
        for (uint32_t i = 0; i < k; ++i) {
            a[i] = (int64_t)(t % p);
            t /= p;
        }
        trim(a);
        bool prim = true;
        for (uint64_t r : rs) {
            Poly x = ppowmod(a, N / r, m, p);
            if (x.size() == 1 && x[0] == 1) {
                prim = false;
                break;
            }
        }
        if (N == 1) prim = (a.size() == 1 && a[0] == 1);
        if (prim) {
            g = a;
            break;
        }
    }
    if (g.empty()) return set_error(QADIC_E_INVALID, "no generator found");
    for (uint32_t i = 0; i < k; ++i) f.gen[i] = i < g.size() ? (uint32_t)g[i] : 0;

    // Antilog table: row e = g^e, row N = zero.
    f.antilog.assign((size_t)order * k, 0);
    Poly x{1};
    for (uint64_t e = 0; e < N; ++e) {
        for (uint32_t i = 0; i < k; ++i) f.antilog[e * k + i] = i < x.size() ? (uint8_t)x[i] : 0;
        x = pmulmod(x, g, m, p);
    }

    // q and n_q: q = 2^s with (2k-1) s <= 51, so that every packed block sum
    // r < q^(2k-1) <= 2^51 satisfies both Eq. 2 (m = 53) and Lemma 1's limit;
    // n_q the largest block with n_q k (p-1)^2 < q (Eq. 2).
    f.log2_q = 51 / (2 * k - 1);
    const uint64_t q = 1ull << f.log2_q;
    const uint64_t step = (uint64_t)k * (p - 1) * (p - 1);
    f.n_q = (uint32_t)std::min<uint64_t>((q - 1) / step, 1u << 30);

    // Eq. 3 with the centred representation: k K h^2 <= 2^31 - 1.
    const uint64_t hh = (uint64_t)f.h * f.h;
    f.k_max_int32 = (int64_t)(((1ull << 31) - 1) / (k * hh));
    // FP32 accumulation: a drained residue (|.| <= 1.5 p, see the tensor-core
    // kernel's drain) plus k K h^2 must stay <= 2^24; 2p is used as margin.
    f.k_chunk_f32 = (int64_t)(((1ull << 24) - 2 * p) / (k * hh));

    // Conversion tables.
    f.log_f64.assign(order, 0.0);
    f.log_centred.assign((size_t)order * k, 0);
    for (uint64_t e = 0; e < order; ++e) {
        uint64_t w = 0;
        for (uint32_t i = 0; i < k; ++i) {
            const uint32_t c = f.antilog[e * k + i];
            w += (uint64_t)c << (f.log2_q * i);
            int32_t cc = (int32_t)c;
            if (p > 2 && cc > (int32_t)f.h) cc -= (int32_t)p;
            f.log_centred[e * k + i] = (int8_t)cc;
        }
        f.log_f64[e] = (double)w;
    }

    // X^(k+t) mod P, t = 0..k-2 (fold of the high product coefficients).
    f.fold.assign((size_t)(k > 1 ? k - 1 : 0) * k, 0);
    for (uint32_t t = 0; t + 1 < k; ++t) {
        Poly xt(k + t + 1, 0);
        xt[k + t] = 1;
        Poly r = pmod(xt, m, p);
        for (uint32_t i = 0; i < k; ++i) f.fold[t * k + i] = i < r.size() ? (uint8_t)r[i] : 0;
    }

    // Thm. 3 tables (k <= 4 so that k bytes pack into 32 bits).  With
    // mu_{2k-2} = u_{2k-2} and mu_i = (u_i - q u_{i+1}) mod p:
    //   L[(u_0..u_{k-1})]      = sum_{i=0}^{k-2} mu_i X^i
    //   H[(u_{k-1}..u_{2k-2})] = (sum_{i=k-1}^{2k-2} mu_i X^i) mod P
    // and the block's field value is L + H.
    if (k <= 4) {
        const int64_t qm = (int64_t)(q % p);
        f.tab_L.assign(order, 0);
        f.tab_H.assign(order, 0);
        std::vector<int64_t> u(k);
        for (uint64_t idx = 0; idx < order; ++idx) {
            uint64_t t = idx;
            for (uint32_t i = 0; i < k; ++i) {
                u[i] = (int64_t)(t % p);
                t /= p;
            }
            uint32_t L = 0;
            for (uint32_t i = 0; i + 1 < k; ++i) {
                const int64_t mu = ((u[i] - qm * u[i + 1]) % (int64_t)p + p) % p;
                L |= (uint32_t)mu << (8 * i);
            }
            f.tab_L[idx] = L;
            // H: u here holds (u_{k-1} .. u_{2k-2}); position j <-> X^(k-1+j).
            Poly hp(2 * k - 1, 0);
            for (uint32_t j = 0; j < k; ++j) {
                const int64_t mu =
                    (j + 1 < k) ? ((u[j] - qm * u[j + 1]) % (int64_t)p + p) % p : u[j];
                hp[k - 1 + j] = mu;
            }
            Poly r = pmod(hp, m, p);
            uint32_t H = 0;
            for (uint32_t i = 0; i < k; ++i) H |= (uint32_t)(i < r.size() ? r[i] : 0) << (8 * i);
            f.tab_H[idx] = H;
        }
    }
    return QADIC_OK;
}

}  // namespace qadic
