/* CPU oracle: the counter-based Rademacher JL sketch Y^T = M^T Q^T (test infrastructure only).
 *
 * M = [W^{1/2} B; D^{1/2}] stacks one row per edge (mesh segment, TSV segment, pad);
 * Q is k x m with entries +-1/sqrt(k).  Entry Q[j][e] takes its sign from the top bit
 * of SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) applied to key XOR (e * 2^32 + j),
 * key = SplitMix64(seed): top bit 0 -> +1, top bit 1 -> -1.  Row e of M has +sqrt(w_e) at the lower node id,
 * -sqrt(w_e) at the higher one; a pad row has +sqrt(g) at its node.
 *
 * This is the plain edge loop; it shares nothing with the CUDA library.
 */
#include <stdint.h>
#include <math.h>

static uint64_t oracle_splitmix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Yt is n x k, row-major, zero on entry.  Edges with w <= 0 contribute nothing. */
void oracle_sketch(int64_t n, int32_t k, uint64_t seed,
                   int64_t m, const int64_t *u, const int64_t *v, const double *w, const int64_t *eid,
                   int64_t np, const int64_t *pu, const double *pw, const int64_t *peid,
                   double *Yt)
{
    (void)n;
    const double rk = 1.0 / sqrt((double)k);
    const uint64_t key = oracle_splitmix64(seed);
    for (int64_t e = 0; e < m; ++e) {
        if (!(w[e] > 0.0)) continue;
        const double s = sqrt(w[e]) * rk;
        double *ru = Yt + u[e] * (int64_t)k;
        double *rv = Yt + v[e] * (int64_t)k;
        for (int32_t j = 0; j < k; ++j) {
            uint64_t h = oracle_splitmix64(key ^ (((uint64_t)eid[e] << 32) | (uint32_t)j));
            double q = (h >> 63) ? -s : s;
            ru[j] += q;
            rv[j] -= q;
        }
    }
    for (int64_t e = 0; e < np; ++e) {
        if (!(pw[e] > 0.0)) continue;
        const double s = sqrt(pw[e]) * rk;
        double *ru = Yt + pu[e] * (int64_t)k;
        for (int32_t j = 0; j < k; ++j) {
            uint64_t h = oracle_splitmix64(key ^ (((uint64_t)peid[e] << 32) | (uint32_t)j));
            ru[j] += (h >> 63) ? -s : s;
        }
    }
}
