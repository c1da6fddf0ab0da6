/*
 * pmc_oracle.c -- CPU FP64 oracle of Progressive Material Caching.
 *
 * TEST INFRASTRUCTURE ONLY (see pmc_oracle.h).  Written for clarity, not speed:
 * one shading point at a time, one node at a time, one table slot at a time.
 */
#include "pmc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ========================================================================== */
/* Published mixers                                                           */
/* ========================================================================== */

/* MurmurHash3 fmix32 (Appleby, public domain): xor-shift / multiply avalanche. */
uint32_t orc_fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

/* MurmurHash3 fmix64 (Appleby, public domain). */
uint64_t orc_fmix64(uint64_t k) {
    k ^= k >> 33;
    k *= 0xFF51AFD7ED558CCDull;
    k ^= k >> 33;
    k *= 0xC4CEB9FE1A85EC53ull;
    k ^= k >> 33;
    return k;
}

/* Output function of SplitMix64 (Steele, Lea & Flood 2014). */
uint64_t orc_splitmix64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* ========================================================================== */
/* Node primitives (the paper leaves them to the renderer; defined here)      */
/* ========================================================================== */

/* Integer lattice hash: the three primes of Teschner et al. 2003 ("Optimized
 * spatial hashing for collision detection of deformable objects") combined by
 * xor, then the MurmurHash3 32-bit finaliser.  Arithmetic is modulo 2^32;
 * negative lattice indices wrap as two's complement. */
uint32_t orc_lattice_hash(int64_t i, int64_t j, uint32_t seed) {
    uint32_t ui = (uint32_t)i;
    uint32_t uj = (uint32_t)j;
    uint32_t h = (ui * 73856093u) ^ (uj * 19349663u) ^ (seed * 83492791u);
    return orc_fmix32(h);
}

/* Perlin's improved-noise interpolant 6t^5 - 15t^4 + 10t^3 (Perlin 2002). */
double orc_fade(double t) {
    return 6.0 * pow(t, 5) - 15.0 * pow(t, 4) + 10.0 * pow(t, 3);
}

/* The 8 unit gradients at multiples of 45 degrees, selected by hash & 7. */
static void gradient(int64_t i, int64_t j, uint32_t seed, double* gx, double* gy) {
    uint32_t k = orc_lattice_hash(i, j, seed) & 7u;
    double ang = (double)k * (M_PI / 4.0);
    *gx = cos(ang);
    *gy = sin(ang);
    /* cos/sin of multiples of pi/4 are 0, +-1 or +-sqrt(1/2); snap the zeros
     * and ones that cos/sin return with a last-bit error. */
    if (fabs(*gx) < 1e-12) *gx = 0.0;
    if (fabs(*gy) < 1e-12) *gy = 0.0;
    if (fabs(fabs(*gx) - 1.0) < 1e-12) *gx = *gx > 0 ? 1.0 : -1.0;
    if (fabs(fabs(*gy) - 1.0) < 1e-12) *gy = *gy > 0 ? 1.0 : -1.0;
}

static double lerp(double a, double b, double t) { return a + (b - a) * t; }

/* 2-D gradient noise (Perlin 1985/2002): a gradient at every lattice point,
 * dotted with the offset to the sample, blended with the quintic fade. */
double orc_perlin(double x, double y, uint32_t seed) {
    double fx0 = floor(x), fy0 = floor(y);
    int64_t ix = (int64_t)fx0, iy = (int64_t)fy0;
    double fx = x - fx0, fy = y - fy0;
    double d[2][2];
    for (int cy = 0; cy < 2; ++cy) {
        for (int cx = 0; cx < 2; ++cx) {
            double gx, gy;
            gradient(ix + cx, iy + cy, seed, &gx, &gy);
            d[cy][cx] = gx * (fx - cx) + gy * (fy - cy);
        }
    }
    double su = orc_fade(fx), sv = orc_fade(fy);
    return lerp(lerp(d[0][0], d[0][1], su), lerp(d[1][0], d[1][1], su), sv);
}

static double clamp01(double x) { return x < 0.0 ? 0.0 : (x > 1.0 ? 1.0 : x); }

/* Fractal Brownian motion: octave k samples noise at frequency scale*lac^k with
 * weight gain^k and seed + k; the weighted sum is normalised by the sum of the
 * weights and mapped to 0.5 + f, clamped to [0, 1]. */
double orc_fbm(double x, double y, double scale, int octaves, double lacunarity,
               double gain, uint32_t seed) {
    double sum = 0.0, norm = 0.0;
    for (int k = 0; k < octaves; ++k) {
        double freq = scale * pow(lacunarity, k);
        double amp = pow(gain, k);
        sum += amp * orc_perlin(x * freq, y * freq, seed + (uint32_t)k);
        norm += amp;
    }
    return clamp01(0.5 + sum / norm);
}

/* Worley (1996) F1: distance to the nearest feature point, one feature point
 * per unit cell at cell + 0.25 + 0.5 * (16-bit fractions of the cell hash).
 * The 0.25 margin makes the 3x3 neighbourhood exact: a point outside it is at
 * least 1.25 away, the own cell's point at most sqrt(2) * 0.75 ~ 1.06. */
double orc_voronoi_f1(double x, double y, uint32_t seed) {
    double fx0 = floor(x), fy0 = floor(y);
    int64_t ix = (int64_t)fx0, iy = (int64_t)fy0;
    double fx = x - fx0, fy = y - fy0;
    double best = INFINITY;
    for (int b = -1; b <= 1; ++b) {
        for (int a = -1; a <= 1; ++a) {
            uint32_t h = orc_lattice_hash(ix + a, iy + b, seed);
            double ox = a + 0.25 + 0.5 * ((double)(h & 0xFFFFu) / 65536.0);
            double oy = b + 0.25 + 0.5 * ((double)(h >> 16) / 65536.0);
            double d2 = (ox - fx) * (ox - fx) + (oy - fy) * (oy - fy);
            if (d2 < best) best = d2;
        }
    }
    return sqrt(best);
}

void orc_eval_node(const orc_node* nd, const double* a, const double* b, const double* c,
                   const double sp[8], double out[3]) {
    const float* p = nd->fp;
    switch (nd->op) {
    case ORC_UV:
        out[0] = sp[0]; out[1] = sp[1]; out[2] = 0.0;
        return;
    case ORC_POSITION:
        out[0] = sp[2]; out[1] = sp[3]; out[2] = sp[4];
        return;
    case ORC_NORMAL:
        out[0] = sp[5]; out[1] = sp[6]; out[2] = sp[7];
        return;
    case ORC_CONST:
        out[0] = p[0]; out[1] = p[1]; out[2] = p[2];
        return;
    case ORC_UV_AFFINE: /* [x'; y'] = [p0 p1; p2 p3] [x; y] + [p4; p5]; not clamped */
        out[0] = (double)p[0] * a[0] + (double)p[1] * a[1] + (double)p[4];
        out[1] = (double)p[2] * a[0] + (double)p[3] * a[1] + (double)p[5];
        out[2] = 0.0;
        return;
    case ORC_FBM: {
        double s = orc_fbm(a[0], a[1], p[0], nd->ip[0], p[1], p[2], (uint32_t)nd->ip[1]);
        out[0] = out[1] = out[2] = s;
        return;
    }
    case ORC_VORONOI: {
        double s = clamp01(orc_voronoi_f1(a[0] * p[0], a[1] * p[0], (uint32_t)nd->ip[1]));
        out[0] = out[1] = out[2] = s;
        return;
    }
    case ORC_CHECKER: {
        int64_t k = (int64_t)floor(a[0] * p[0]) + (int64_t)floor(a[1] * p[0]);
        const float* col = (k & 1) ? &p[4] : &p[1];
        for (int i = 0; i < 3; ++i) out[i] = clamp01(col[i]);
        return;
    }
    case ORC_RAMP: {
        int ns = nd->ip[0];
        double t = clamp01(a[0]);
        double res[3];
        if (t <= p[0]) {
            for (int i = 0; i < 3; ++i) res[i] = p[4 + i];
        } else if (t >= p[ns - 1]) {
            for (int i = 0; i < 3; ++i) res[i] = p[4 + 3 * (ns - 1) + i];
        } else {
            for (int k = 0; k + 1 < ns; ++k) {
                if (t < p[k + 1]) {
                    double w = (t - p[k]) / ((double)p[k + 1] - (double)p[k]);
                    for (int i = 0; i < 3; ++i)
                        res[i] = lerp(p[4 + 3 * k + i], p[4 + 3 * (k + 1) + i], w);
                    break;
                }
            }
        }
        for (int i = 0; i < 3; ++i) out[i] = clamp01(res[i]);
        return;
    }
    case ORC_MIX: {
        double f = clamp01(c ? c[0] : (double)p[0]);
        for (int i = 0; i < 3; ++i) out[i] = clamp01(lerp(a[i], b[i], f));
        return;
    }
    case ORC_ADD:
        for (int i = 0; i < 3; ++i) out[i] = clamp01(a[i] + b[i]);
        return;
    case ORC_MUL:
        for (int i = 0; i < 3; ++i) out[i] = clamp01(a[i] * b[i]);
        return;
    case ORC_POW:
        for (int i = 0; i < 3; ++i) {
            double x = a[i] > 0.0 ? a[i] : 0.0;
            out[i] = clamp01(pow(x, (double)p[0]));
        }
        return;
    case ORC_FACING: {
        double s = clamp01(fabs(a[0] * p[0] + a[1] * p[1] + a[2] * p[2]));
        out[0] = out[1] = out[2] = s;
        return;
    }
    default:
        out[0] = out[1] = out[2] = 0.0;
        return;
    }
}

/* ========================================================================== */
/* Descriptor and hashes                                                      */
/* ========================================================================== */

/* Texel index on a virtual texture of 2^level texels per axis (Sec. 3.1):
 * clamp u to [0, 1] (NaN to 0), then floor(u * 2^level), with u = 1 mapped to
 * the last texel. */
uint32_t orc_texel(float u, uint32_t level) {
    double x = (double)u;
    if (!(x >= 0.0)) x = 0.0;
    if (x > 1.0) x = 1.0;
    double r = ldexp(1.0, (int)level);
    double t = floor(x * r);
    if (t > r - 1.0) t = r - 1.0;
    return (uint32_t)t;
}

/* Mip level of the virtual texture from the ray-cone footprint (Sec. 3.1, Eq. 1):
 * lambda = -log2(min(|g1|, |g2|)), g1 and g2 the texture-coordinate gradients along the
 * axes of the footprint ellipse.  Readings: each squared norm is formed in FP32 with
 * every product and the sum rounded to nearest (the decision is taken in the precision
 * the inputs have); the level is the floor of Eq. 1, so that a texel is at least as wide
 * as the footprint; the offset of the discussion (Sec. 4) is added; the result is
 * clamped to [0, 13].  A zero footprint gives the finest level, an infinite or NaN one
 * the coarsest. */
int32_t orc_level(float g1u, float g1v, float g2u, float g2v, int32_t offset) {
    const float a = g1u * g1u, b = g1v * g1v, c = g2u * g2u, d = g2v * g2v;   /* no contraction */
    const float s1 = a + b, s2 = c + d;
    double lam;
    if (isnan(s1) || isnan(s2)) {
        lam = -INFINITY;
    } else {
        const double m = sqrt((double)(s1 < s2 ? s1 : s2));   /* min(|g1|, |g2|) */
        lam = m == 0.0 ? INFINITY : floor(-log2(m));
    }
    lam += (double)offset;
    if (!(lam > 0.0)) return 0;
    if (lam > 13.0) return 13;
    return (int32_t)lam;
}

/* The 32-bit encoding of a cached value (Sec. 3.3, Alg. 1 "Encode"): the paper packs the
 * second hash and the encoded value into one 64-bit word for a single compare-and-swap
 * but does not name the format.  Reading: the shared-exponent format of OpenGL's
 * EXT_texture_shared_exponent (RGB9E5): three 9-bit mantissas and one 5-bit exponent
 * with bias 15, bits r 0-8, g 9-17, b 18-26, exponent 27-31; components clamped to
 * [0, 511/512 * 2^16] (NaN to 0), each rounded to nearest with ties up at the exponent of
 * the largest.  Written from the format's definition, in FP64 on the FP32 value. */
uint32_t orc_rgb9e5_encode(float r, float g, float b) {
    const double maxv = 511.0 / 512.0 * 65536.0;
    double c[3] = {r, g, b};
    double mx = 0.0;
    for (int k = 0; k < 3; ++k) {
        if (!(c[k] > 0.0)) c[k] = 0.0;   /* negative and NaN */
        if (c[k] > maxv) c[k] = maxv;
        if (c[k] > mx) mx = c[k];
    }
    int fl = -16;                       /* max(-B - 1, floor(log2(max))) */
    if (mx > 0.0) {
        int e;
        frexp(mx, &e);                  /* mx = m 2^e, m in [0.5, 1): floor(log2 mx) = e - 1 */
        if (e - 1 > fl) fl = e - 1;
    }
    int ex = fl + 16;                   /* + 1 + B */
    if (floor(ldexp(mx, 24 - ex) + 0.5) == 512.0) ex += 1;
    uint32_t code = (uint32_t)ex << 27;
    for (int k = 0; k < 3; ++k) code |= (uint32_t)floor(ldexp(c[k], 24 - ex) + 0.5) << (9 * k);
    return code;
}

void orc_rgb9e5_decode(uint32_t code, float out[3]) {
    const int ex = (int)(code >> 27);
    for (int k = 0; k < 3; ++k) out[k] = (float)ldexp((double)((code >> (9 * k)) & 511u), ex - 24);
}

/* Descriptor (Sec. 3.1): material ID, node ID (index in the network as given),
 * mip level lambda, texel indices, packed as
 * mat<<48 | node<<32 | level<<26 | iu<<13 | iv. */
uint64_t orc_key(uint32_t mat, uint32_t node, uint32_t level, float u, float v) {
    uint64_t iu = orc_texel(u, level), iv = orc_texel(v, level);
    return ((uint64_t)mat << 48) | ((uint64_t)node << 32) | ((uint64_t)level << 26) |
           (iu << 13) | iv;
}

/* Voxel index of one coordinate on a grid of 2^-level world units: floor(p 2^level)
 * clamped to [-512, 511], offset to [0, 1023].  p 2^level is exact in FP32 (a power of two
 * scale); NaN takes the lowest voxel. */
uint32_t orc_voxel(float p, uint32_t level) {
    float x = p * ldexpf(1.0f, (int)level);
    if (!(x >= -512.0f)) x = -512.0f;
    if (x > 511.0f) x = 511.0f;
    return (uint32_t)((int32_t)floorf(x) + 512);
}

/* World-position descriptor (the extension Sec. 3.1 and Sec. 5 suggest): material ID,
 * node ID and the voxel of the shading point's position, packed as
 * mat<<48 | node<<32 | 1<<31 | ix<<20 | iy<<10 | iz (bit 31 tells it from a UV key). */
uint64_t orc_key_pos(uint32_t mat, uint32_t node, uint32_t level, float px, float py, float pz) {
    return ((uint64_t)mat << 48) | ((uint64_t)node << 32) | (1ull << 31) |
           ((uint64_t)orc_voxel(px, level) << 20) | ((uint64_t)orc_voxel(py, level) << 10) |
           (uint64_t)orc_voxel(pz, level);
}

/* Hash of Alg. 1 (cell selection): SplitMix64 output function of the key. */
uint64_t orc_hash1(uint64_t key) { return orc_splitmix64_mix(key); }

/* Hash2 of Alg. 1 (entry check): upper 32 bits of fmix64(key xor golden gamma);
 * 0 is reserved for an empty entry and maps to 1. */
uint32_t orc_hash2(uint64_t key) {
    uint32_t h = (uint32_t)(orc_fmix64(key ^ 0x9E3779B97F4A7C15ull) >> 32);
    return h == 0 ? 1u : h;
}

/* Descriptor, cell and check value (Sec. 3.1; Alg. 1) of n (material, node, u, v) tuples
 * at one level: a loop over orc_key, orc_hash1 mod n_cells and orc_hash2, for comparisons
 * over many tuples. */
void orc_address_batch(const uint32_t* mat, const uint32_t* node, const float* u, const float* v,
                       uint64_t n, uint32_t level, uint64_t n_cells, uint64_t* key, uint64_t* cell,
                       uint32_t* h2) {
    for (uint64_t i = 0; i < n; ++i) {
        key[i] = orc_key(mat[i], node[i], level, u[i], v[i]);
        cell[i] = orc_hash1(key[i]) % n_cells;
        h2[i] = orc_hash2(key[i]);
    }
}

/* The two 64-bit mixers behind Hash and Hash2 over n keys: h1 = SplitMix64's output
 * function of the key, m2 = fmix64(key xor golden gamma), whose upper half is Hash2. */
void orc_mix_batch(const uint64_t* key, uint64_t n, uint64_t* h1, uint64_t* m2) {
    for (uint64_t i = 0; i < n; ++i) {
        h1[i] = orc_splitmix64_mix(key[i]);
        m2[i] = orc_fmix64(key[i] ^ 0x9E3779B97F4A7C15ull);
    }
}

/* ========================================================================== */
/* Network analysis (Sec. 3)                                                  */
/* ========================================================================== */

static int n_required_inputs(uint32_t op, int* optional) {
    *optional = 0;
    switch (op) {
    case ORC_UV: case ORC_POSITION: case ORC_NORMAL: case ORC_CONST:
        return 0;
    case ORC_UV_AFFINE: case ORC_FBM: case ORC_VORONOI: case ORC_CHECKER:
    case ORC_RAMP: case ORC_POW: case ORC_FACING:
        return 1;
    case ORC_MIX:
        *optional = 1;
        return 2;
    case ORC_ADD: case ORC_MUL:
        return 2;
    default:
        return -1;
    }
}

/* x is 2^e with -20 <= e <= 20. */
static int power_of_two_scale(float x) {
    int e;
    const double m = frexp((double)x, &e);
    return m == 0.5 && e - 1 >= -20 && e - 1 <= 20;
}

/* The checker is the one discontinuous primitive: its colour flips where x s or y s
 * crosses an integer, so FP32 and FP64 may disagree by a whole colour next to an edge
 * unless the argument is exact in FP32.  It is when x and y come from the UV or the
 * position input, either directly or through an affine map that only scales each axis by
 * a power of two (no rotation, no offset), and s is a power of two: every product is then
 * a power-of-two scaling, exact for any input of magnitude 0 or at least 2^-100. */
static int exact_checker(const orc_node* nodes, const orc_node* nd) {
    if (!power_of_two_scale(nd->fp[0])) return 0;
    const orc_node* src = &nodes[nd->in[0]];
    if (src->op == ORC_UV || src->op == ORC_POSITION) return 1;
    if (src->op != ORC_UV_AFFINE) return 0;
    const uint32_t in = nodes[src->in[0]].op;
    const float* a = src->fp;
    return (in == ORC_UV || in == ORC_POSITION) && power_of_two_scale(a[0]) && power_of_two_scale(a[3]) &&
           a[1] == 0.0f && a[2] == 0.0f && a[4] == 0.0f && a[5] == 0.0f;
}

int orc_validate(const orc_node* nodes, uint32_t n) {
    if (n == 0 || n > 65535u) return ORC_ERR_ARG;
    for (uint32_t i = 0; i < n; ++i) {
        const orc_node* nd = &nodes[i];
        int opt;
        int req = n_required_inputs(nd->op, &opt);
        if (req < 0) return ORC_ERR_ARG;
        for (int k = 0; k < 4; ++k) {
            int32_t x = nd->in[k];
            if (k < req) {
                if (x < 0 || (uint32_t)x >= i) return ORC_ERR_ARG;
            } else if (k < req + opt) {
                if (x < -1 || (x >= 0 && (uint32_t)x >= i)) return ORC_ERR_ARG;
            } else if (x != -1) {
                return ORC_ERR_ARG;
            }
        }
        if (nd->op == ORC_FBM && (nd->ip[0] < 1 || nd->ip[0] > 16)) return ORC_ERR_ARG;
        if (nd->op == ORC_RAMP) {
            int ns = nd->ip[0];
            if (ns < 2 || ns > 4) return ORC_ERR_ARG;
            for (int k = 0; k < ns; ++k) {
                if (!(nd->fp[k] >= 0.0f && nd->fp[k] <= 1.0f)) return ORC_ERR_ARG;
                if (k > 0 && nd->fp[k] < nd->fp[k - 1]) return ORC_ERR_ARG;
            }
        }
        if (nd->op == ORC_POW && !(nd->fp[0] > 0.0f)) return ORC_ERR_ARG;
        if (nd->op == ORC_CHECKER && !exact_checker(nodes, nd)) return ORC_ERR_ARG;
    }
    return ORC_OK;
}

static int is_input_op(uint32_t op) {
    return op == ORC_UV || op == ORC_POSITION || op == ORC_NORMAL || op == ORC_CONST;
}

/* Marks the sub-graph of node r (r and everything it reads) in mark[]. */
static void mark_subgraph(const orc_node* nodes, uint32_t r, uint8_t* mark) {
    mark[r] = 1;
    for (int32_t i = (int32_t)r; i >= 0; --i) {
        if (!mark[i]) continue;
        for (int k = 0; k < 4; ++k)
            if (nodes[i].in[k] >= 0) mark[nodes[i].in[k]] = 1;
    }
}

/* Class of a node whose inputs have classes a and b: constants change nothing, two
 * different shading-point dependences (UV with position, or anything with SP) make it
 * SP (no descriptor of one kind identifies it). */
static int join_class(int a, int b) {
    if (a == b || b == ORC_CLS_CONST) return a;
    if (a == ORC_CLS_CONST) return b;
    return ORC_CLS_SP;
}

/* The node cost model of the library's interface: FP32 operations of one evaluation of a
 * node, a fused multiply-add counted as 2 (UV, POSITION, NORMAL, CONST 0; UV_AFFINE 8; FBM
 * 4 + 47 per octave; VORONOI 99; CHECKER 4; RAMP 23; MIX 17; ADD and MUL 9; POW 18; FACING 8). */
uint32_t orc_node_cost(const orc_node* nd) {
    switch (nd->op) {
    case ORC_UV_AFFINE: return 8;
    case ORC_FBM: return 4 + 47 * (uint32_t)nd->ip[0];
    case ORC_VORONOI: return 99;
    case ORC_CHECKER: return 4;
    case ORC_RAMP: return 23;
    case ORC_MIX: return 17;
    case ORC_ADD: case ORC_MUL: return 9;
    case ORC_POW: return 18;
    case ORC_FACING: return 8;
    default: return 0;
    }
}

/* Dependence classes and cacheable roots.
 *   class(UV input) = UV; class(normal) = SP; class(const) = CONST;
 *   class(position) = POS with the world-position descriptor, else SP;
 *   any other node joins the classes of its inputs (join_class).
 * A node is a cacheable root when it is reachable from the output, has class
 * UV (or POS), is not a bare input, is the output or feeds some SP-class node
 * ("the highest possible level", Sec. 3), its sub-graph holds at least
 * min_root_nodes nodes that are not inputs or constants, and the sub-graph's nodes
 * (each once) cost at least min_root_cost by orc_node_cost.  is_root[i] = 1 for a
 * root with a UV descriptor, 2 for one with a world-position descriptor. */
int orc_analyze_cost(const orc_node* nodes, uint32_t n, uint32_t min_root_nodes, uint32_t min_root_cost,
                     int pos_desc, int32_t* cls, uint8_t* is_root, uint32_t* n_roots) {
    if (orc_validate(nodes, n) != ORC_OK) return ORC_ERR_ARG;
    for (uint32_t i = 0; i < n; ++i) {
        const orc_node* nd = &nodes[i];
        int c;
        if (nd->op == ORC_UV) c = ORC_CLS_UV;
        else if (nd->op == ORC_POSITION) c = pos_desc ? ORC_CLS_POS : ORC_CLS_SP;
        else if (nd->op == ORC_NORMAL) c = ORC_CLS_SP;
        else if (nd->op == ORC_CONST) c = ORC_CLS_CONST;
        else {
            c = ORC_CLS_CONST;
            for (int k = 0; k < 4; ++k)
                if (nd->in[k] >= 0) c = join_class(c, cls[nd->in[k]]);
        }
        cls[i] = c;
    }
    uint8_t* reach = (uint8_t*)calloc(n, 1);
    uint8_t* feeds_sp = (uint8_t*)calloc(n, 1);
    uint8_t* mark = (uint8_t*)malloc(n);
    mark_subgraph(nodes, n - 1, reach);
    for (uint32_t i = 0; i < n; ++i) {
        if (!reach[i] || cls[i] != ORC_CLS_SP) continue;
        for (int k = 0; k < 4; ++k)
            if (nodes[i].in[k] >= 0) feeds_sp[nodes[i].in[k]] = 1;
    }
    uint32_t nr = 0;
    for (uint32_t i = 0; i < n; ++i) {
        is_root[i] = 0;
        if (!reach[i] || (cls[i] != ORC_CLS_UV && cls[i] != ORC_CLS_POS)) continue;
        if (nodes[i].op == ORC_UV || nodes[i].op == ORC_POSITION) continue;
        if (!(i == n - 1 || feeds_sp[i])) continue;
        memset(mark, 0, n);
        mark_subgraph(nodes, i, mark);
        uint32_t work = 0;
        uint64_t cost = 0;
        for (uint32_t j = 0; j <= i; ++j) {
            if (!mark[j]) continue;
            if (!is_input_op(nodes[j].op)) ++work;
            cost += orc_node_cost(&nodes[j]);
        }
        if (work < min_root_nodes || cost < min_root_cost) continue;
        is_root[i] = cls[i] == ORC_CLS_POS ? 2 : 1;
        ++nr;
    }
    *n_roots = nr;
    free(reach);
    free(feeds_sp);
    free(mark);
    return ORC_OK;
}

int orc_analyze_desc(const orc_node* nodes, uint32_t n, uint32_t min_root_nodes, int pos_desc,
                     int32_t* cls, uint8_t* is_root, uint32_t* n_roots) {
    return orc_analyze_cost(nodes, n, min_root_nodes, 0, pos_desc, cls, is_root, n_roots);
}

int orc_analyze(const orc_node* nodes, uint32_t n, uint32_t min_root_nodes,
                int32_t* cls, uint8_t* is_root, uint32_t* n_roots) {
    return orc_analyze_desc(nodes, n, min_root_nodes, 0, cls, is_root, n_roots);
}

static const double* input_value(const orc_node* nd, int k, const double* val) {
    return nd->in[k] >= 0 ? &val[3 * nd->in[k]] : NULL;
}

int orc_eval_point_nocache(const orc_node* nodes, uint32_t n, const double sp[8],
                           double rgb[3]) {
    if (orc_validate(nodes, n) != ORC_OK) return ORC_ERR_ARG;
    double* val = (double*)calloc(3 * (size_t)n, sizeof(double));
    uint8_t* reach = (uint8_t*)calloc(n, 1);
    mark_subgraph(nodes, n - 1, reach);
    for (uint32_t i = 0; i < n; ++i) {
        if (!reach[i]) continue;
        orc_eval_node(&nodes[i], input_value(&nodes[i], 0, val), input_value(&nodes[i], 1, val),
                      input_value(&nodes[i], 2, val), sp, &val[3 * i]);
    }
    for (int k = 0; k < 3; ++k) rgb[k] = val[3 * (n - 1) + k];
    free(val);
    free(reach);
    return ORC_OK;
}

/* ========================================================================== */
/* Progressive cache: sequential emulation of the bulk-synchronous update      */
/* ========================================================================== */

typedef struct {
    orc_node* nodes;
    uint32_t n;
    uint8_t* is_root;
    uint32_t n_roots;
    uint32_t* roots; /* ascending node IDs */
    double* surr_theta; /* learned surrogate of node surr_node, or NULL */
    uint32_t surr_node;
    int surr_bf16;
} orc_mat;

struct orc_cache {
    uint64_t n_cells;
    uint32_t n_entries;
    uint32_t level;        /* every point's level when no gradients are given */
    int32_t level_offset;  /* added to the ray-cone level (Sec. 4) */
    int alg1;              /* the paper's concurrent update, serialised point by point */
    int replace;           /* replacement by visibility class (Sec. 5), else keep-first */
    int threads;           /* host threads of orc_run_batch (1 = one point after another) */
    int close_at_lookup;   /* replacement: drop a value as full at lookup when its full cell
                              holds no class larger than its own (1, the default); 0 = let
                              every such value reach the sequential insert */
    int32_t pos_level;     /* world-position descriptor: voxels of 2^-pos_level; -1 = off */
    uint32_t min_root_nodes;
    uint32_t min_root_cost;  /* cost threshold of a cacheable node's sub-graph (0 = none) */
    int off;
    uint32_t* h2;  /* n_cells * n_entries, 0 = empty */
    float* rgb;    /* 3 per slot */
    uint8_t* cls;  /* visibility class of each slot's entry (replacement policy only) */
    orc_mat* mats;
    uint32_t n_mats;
    orc_hash_override_fn hook;
    uint64_t stats[ORC_NSTATS];
};

orc_cache* orc_cache_new(uint64_t n_cells, uint32_t n_entries, uint32_t level,
                         uint32_t min_root_nodes, int cache_off) {
    if (level > 13) return NULL;
    orc_cache* c = (orc_cache*)calloc(1, sizeof(orc_cache));
    c->n_cells = n_cells;
    c->n_entries = n_entries;
    c->level = level;
    c->min_root_nodes = min_root_nodes;
    c->off = cache_off || n_cells == 0 || n_entries == 0;
    size_t slots = c->off ? 0 : (size_t)n_cells * n_entries;
    c->h2 = (uint32_t*)calloc(slots ? slots : 1, sizeof(uint32_t));
    c->rgb = (float*)calloc(slots ? 3 * slots : 1, sizeof(float));
    c->cls = (uint8_t*)calloc(slots ? slots : 1, 1);
    c->pos_level = -1;
    c->close_at_lookup = 1;
    c->threads = 1;
    return c;
}

static void free_mats(orc_cache* c) {
    for (uint32_t m = 0; m < c->n_mats; ++m) {
        free(c->mats[m].surr_theta);
        free(c->mats[m].nodes);
        free(c->mats[m].is_root);
        free(c->mats[m].roots);
    }
    free(c->mats);
    c->mats = NULL;
    c->n_mats = 0;
}

void orc_cache_free(orc_cache* c) {
    if (!c) return;
    free_mats(c);
    free(c->h2);
    free(c->rgb);
    free(c->cls);
    free(c);
}

int orc_cache_set_materials(orc_cache* c, uint32_t n_mats, const orc_node* const* mat_nodes,
                            const uint32_t* n_nodes) {
    if (n_mats > 65536u) return ORC_ERR_ARG;
    free_mats(c);
    c->mats = (orc_mat*)calloc(n_mats ? n_mats : 1, sizeof(orc_mat));
    c->n_mats = n_mats;
    for (uint32_t m = 0; m < n_mats; ++m) {
        uint32_t n = n_nodes[m];
        orc_mat* M = &c->mats[m];
        if (orc_validate(mat_nodes[m], n) != ORC_OK) {
            free_mats(c);
            return ORC_ERR_ARG;
        }
        M->n = n;
        M->nodes = (orc_node*)malloc(n * sizeof(orc_node));
        memcpy(M->nodes, mat_nodes[m], n * sizeof(orc_node));
        M->is_root = (uint8_t*)calloc(n, 1);
        int32_t* cls = (int32_t*)malloc(n * sizeof(int32_t));
        orc_analyze_cost(M->nodes, n, c->min_root_nodes, c->min_root_cost, c->pos_level >= 0, cls, M->is_root,
                         &M->n_roots);
        free(cls);
        M->roots = (uint32_t*)malloc((M->n_roots ? M->n_roots : 1) * sizeof(uint32_t));
        uint32_t r = 0;
        for (uint32_t i = 0; i < n; ++i)
            if (M->is_root[i]) M->roots[r++] = i;
    }
    return ORC_OK;
}

void orc_cache_set_hash_override(orc_cache* c, orc_hash_override_fn fn) { c->hook = fn; }

void orc_cache_set_level_offset(orc_cache* c, int32_t offset) { c->level_offset = offset; }

void orc_cache_set_alg1(orc_cache* c, int on) { c->alg1 = on != 0; }

void orc_cache_set_replacement(orc_cache* c, int on) { c->replace = on != 0; }

void orc_cache_set_close_at_lookup(orc_cache* c, int on) { c->close_at_lookup = on != 0; }

void orc_cache_set_min_root_cost(orc_cache* c, uint32_t cost) { c->min_root_cost = cost; }

void orc_cache_set_threads(orc_cache* c, int threads) { c->threads = threads > 1 ? threads : 1; }

void orc_cache_set_position_level(orc_cache* c, int32_t level) { c->pos_level = level; }

void orc_cache_reset(orc_cache* c) {
    size_t slots = c->off ? 0 : (size_t)c->n_cells * c->n_entries;
    if (slots) {
        memset(c->h2, 0, slots * sizeof(uint32_t));
        memset(c->rgb, 0, 3 * slots * sizeof(float));
        memset(c->cls, 0, slots);
    }
    memset(c->stats, 0, sizeof(c->stats));
}

uint32_t orc_cache_n_roots(const orc_cache* c, uint32_t mat) {
    return mat < c->n_mats ? c->mats[mat].n_roots : 0;
}

void orc_cache_roots(const orc_cache* c, uint32_t mat, uint32_t* out) {
    if (mat >= c->n_mats) return;
    for (uint32_t r = 0; r < c->mats[mat].n_roots; ++r) out[r] = c->mats[mat].roots[r];
}

/* bfloat16 nearest (ties to even) of the float32 nearest to x, as a double */
static double bf16(double x) {
    float f = (float)x;
    uint32_t b;
    memcpy(&b, &f, 4);
    b = (b + 0x7FFFu + ((b >> 16) & 1u)) & 0xFFFF0000u;
    memcpy(&f, &b, 4);
    return (double)f;
}

void orc_mlp_forward(const double* th, double u, double v, int use_bf16, double y[3]) {
    double g[64], h1[64], h2[64];
    for (int k = 0; k < 16; ++k) {
        const double a = M_PI * (double)(k + 1);
        g[k] = sin(a * u);
        g[16 + k] = cos(a * u);
        g[32 + k] = sin(a * v);
        g[48 + k] = cos(a * v);
    }
    if (use_bf16)
        for (int k = 0; k < 64; ++k) g[k] = bf16(g[k]);
    const double* W1 = th;
    const double* b1 = th + 4096;
    const double* W2 = th + 4160;
    const double* b2 = th + 8256;
    const double* W3 = th + 8320;
    const double* b3 = th + 8512;
    for (int o = 0; o < 64; ++o) {
        double z = b1[o];
        for (int i = 0; i < 64; ++i) z += g[i] * (use_bf16 ? bf16(W1[i * 64 + o]) : W1[i * 64 + o]);
        h1[o] = z > 0.0 ? z : 0.0;
        if (use_bf16) h1[o] = bf16(h1[o]);
    }
    for (int o = 0; o < 64; ++o) {
        double z = b2[o];
        for (int i = 0; i < 64; ++i) z += h1[i] * (use_bf16 ? bf16(W2[i * 64 + o]) : W2[i * 64 + o]);
        h2[o] = z > 0.0 ? z : 0.0;
        if (use_bf16) h2[o] = bf16(h2[o]);
    }
    for (int o = 0; o < 3; ++o) {
        double z = b3[o];
        for (int i = 0; i < 64; ++i) z += h2[i] * (use_bf16 ? bf16(W3[i * 3 + o]) : W3[i * 3 + o]);
        y[o] = z;
    }
}

int orc_cache_set_surrogate(orc_cache* c, uint32_t mat, uint32_t node, const double* theta, int use_bf16) {
    if (mat >= c->n_mats) return ORC_ERR_ARG;
    orc_mat* M = &c->mats[mat];
    free(M->surr_theta);
    M->surr_theta = NULL;
    if (!theta) return ORC_OK;
    if (node >= M->n || !M->is_root[node]) return ORC_ERR_ARG;
    M->surr_theta = (double*)malloc(ORC_MLP_PARAMS * sizeof(double));
    memcpy(M->surr_theta, theta, ORC_MLP_PARAMS * sizeof(double));
    M->surr_node = node;
    M->surr_bf16 = use_bf16;
    return ORC_OK;
}

static void cell_and_check(const orc_cache* c, uint64_t key, uint64_t* cell, uint32_t* h2) {
    if (c->hook) {
        c->hook(key, c->n_cells, cell, h2);
        return;
    }
    *cell = orc_hash1(key) % c->n_cells;
    *h2 = orc_hash2(key);
}

/* Scan of one cell as in Alg. 1: the first entry whose stored hash equals h2
 * (found) or is 0 (empty).  Returns 1 = found, 0 = empty, -1 = cell full;
 * *slot receives the entry index. */
static int scan_cell(const orc_cache* c, uint64_t cell, uint32_t h2, uint64_t* slot) {
    for (uint32_t i = 0; i < c->n_entries; ++i) {
        uint64_t s = cell * c->n_entries + i;
        if (c->h2[s] == h2) { *slot = s; return 1; }
        if (c->h2[s] == 0) { *slot = s; return 0; }
    }
    return -1;
}

typedef struct {
    uint64_t cell;
    uint32_t h2;
    float rgb[3];
    uint8_t vis;   /* visibility class of the inserting point */
} orc_candidate;

/* Replacement policy (the prioritisation that Sec. 5 proposes as future work): a full
 * cell gives up the entry of the least important class, provided that class is less
 * important than the newcomer's (a larger class number = more bounces away from the
 * camera).  Returns the slot to overwrite, or -1 when every entry is at least as
 * important as the newcomer.  Among entries of the same class the first one goes. */
static int64_t replacement_victim(const orc_cache* c, uint64_t cell, uint8_t vis) {
    int64_t victim = -1;
    uint8_t worst = vis;
    for (uint32_t i = 0; i < c->n_entries; ++i) {
        uint64_t s = cell * c->n_entries + i;
        if (c->cls[s] > worst) {
            worst = c->cls[s];
            victim = (int64_t)s;
        }
    }
    return victim;
}

/* Inserts candidates one at a time in the given order (Alg. 1 serialised: the
 * compare-and-swap on an empty entry always succeeds; the first value is kept).  With the
 * paper's concurrent update the stored value is the 32-bit encoding of the value, and a
 * hit returns its decoding. */
static void insert_candidates(orc_cache* c, const orc_candidate* cand, size_t n_cand) {
    for (size_t q = 0; q < n_cand; ++q) {
        uint64_t slot;
        int r = scan_cell(c, cand[q].cell, cand[q].h2, &slot);
        if (r == 1) {
            c->stats[5]++;
        } else if (r == 0) {
            c->h2[slot] = cand[q].h2;
            c->cls[slot] = cand[q].vis;
            if (c->alg1)
                orc_rgb9e5_decode(orc_rgb9e5_encode(cand[q].rgb[0], cand[q].rgb[1], cand[q].rgb[2]),
                                  &c->rgb[3 * slot]);
            else
                for (int k = 0; k < 3; ++k) c->rgb[3 * slot + k] = cand[q].rgb[k];
            c->stats[4]++;
        } else {
            int64_t v = c->replace ? replacement_victim(c, cand[q].cell, cand[q].vis) : -1;
            if (v >= 0) {
                /* the evicted entry's descriptor misses from now on; the cell stays
                 * full, so occupied slots still form a prefix */
                c->h2[v] = cand[q].h2;
                c->cls[v] = cand[q].vis;
                for (int k = 0; k < 3; ++k) c->rgb[3 * (uint64_t)v + k] = cand[q].rgb[k];
                c->stats[9]++;
            } else {
                c->stats[6]++;
            }
        }
    }
}

/* The inputs and outputs of one batch, as orc_run_batch receives them. */
typedef struct {
    uint64_t n;
    const float *u, *v;
    const uint32_t* mat;
    const float *px, *py, *pz, *nx, *ny, *nz;
    double* rgb;
    uint16_t* hits;
    uint32_t* evaluated;
    uint64_t* probe_key;
    uint64_t* probe_cell;
    uint32_t* probe_h2;
    uint8_t* probe_hit;
    const float *g1u, *g1v, *g2u, *g2v;
    const uint8_t* vis;
} orc_batch;

/* Scratch of one range of points: per-node values and flags, the candidates the range
 * produced (in point order) and its counters. */
typedef struct {
    double* val;
    uint8_t* hit;
    double* hitval;
    uint8_t* needed;
    uint64_t* rcell;
    uint32_t* rh2;
    uint8_t* rclosed;   /* replacement: the cell cannot take the value */
    orc_candidate* cand;
    size_t n_cand, cand_cap;
    uint64_t stats[ORC_NSTATS];
    int status;
} orc_work;

static void work_init(orc_work* w, uint32_t max_n) {
    memset(w, 0, sizeof(*w));
    w->val = (double*)malloc(3 * (size_t)max_n * sizeof(double));
    w->hit = (uint8_t*)malloc(max_n);
    w->hitval = (double*)malloc(3 * (size_t)max_n * sizeof(double));
    w->needed = (uint8_t*)malloc(max_n);
    w->rcell = (uint64_t*)malloc((size_t)max_n * sizeof(uint64_t));
    w->rh2 = (uint32_t*)malloc((size_t)max_n * sizeof(uint32_t));
    w->rclosed = (uint8_t*)malloc(max_n);
    w->cand_cap = 1024;
    w->cand = (orc_candidate*)malloc(w->cand_cap * sizeof(orc_candidate));
    w->status = ORC_OK;
}

static void work_free(orc_work* w) {
    free(w->val);
    free(w->hit);
    free(w->hitval);
    free(w->needed);
    free(w->rcell);
    free(w->rh2);
    free(w->rclosed);
    free(w->cand);
}

/* Phase L and evaluation of point i: every point sees the table as it was when the batch
 * started (with the paper's concurrent update, as the earlier points of the batch left
 * it).  probe0: the point's first entry in the probe_* arrays. */
static void process_point(orc_cache* c, const orc_batch* B, uint64_t i, uint64_t probe0, orc_work* w) {
    const uint64_t n = B->n;
    if (B->mat[i] >= c->n_mats) {
        w->status = ORC_ERR_BADMAT;
        B->rgb[i] = B->rgb[n + i] = B->rgb[2 * n + i] = 0.0;
        if (B->hits) B->hits[i] = 0;
        if (B->evaluated) B->evaluated[i] = 0;
        return;
    }
    const uint32_t mi = B->mat[i];
    const orc_mat* M = &c->mats[mi];
    const double sp[8] = {B->u[i], B->v[i], B->px[i], B->py[i], B->pz[i], B->nx[i], B->ny[i], B->nz[i]};
    /* the point's mip level: from its ray-cone gradients (Eq. 1) if given */
    const uint32_t level =
        B->g1u ? (uint32_t)orc_level(B->g1u[i], B->g1v[i], B->g2u[i], B->g2v[i], c->level_offset) : c->level;
    uint32_t n_hit = 0;
    uint64_t probe = probe0;
    memset(w->hit, 0, M->n);
    for (uint32_t r = 0; r < M->n_roots; ++r) {
        uint32_t node = M->roots[r];
        /* a node with a learned surrogate takes the network's value, no lookup */
        const int surr = M->surr_theta && node == M->surr_node;
        if (surr) {
            double y[3];
            orc_mlp_forward(M->surr_theta, B->u[i], B->v[i], M->surr_bf16, y);
            w->hit[node] = 1;
            for (int k = 0; k < 3; ++k) w->hitval[3 * node + k] = clamp01(y[k]);
        }
        if (c->off) continue;
        uint64_t key = M->is_root[node] == 2
                           ? orc_key_pos(mi, node, (uint32_t)c->pos_level, B->px[i], B->py[i], B->pz[i])
                           : orc_key(mi, node, level, B->u[i], B->v[i]);
        uint64_t cell, slot;
        uint32_t h2;
        cell_and_check(c, key, &cell, &h2);
        w->rcell[node] = cell;
        w->rh2[node] = h2;
        int found = 0;
        w->rclosed[node] = 0;
        if (!surr) {
            const int sc = scan_cell(c, cell, h2, &slot);
            found = sc == 1;
            /* Replacement: a cell that is full of entries whose classes are all at most
             * the point's own can never take its value in this batch (classes in a
             * full cell only decrease), so the value is dropped as full at lookup. */
            if (sc < 0 && c->replace && c->close_at_lookup) {
                const uint8_t q = B->vis ? B->vis[i] : 0;
                uint8_t mx = 0;
                for (uint32_t e = 0; e < c->n_entries; ++e)
                    if (c->cls[cell * c->n_entries + e] > mx) mx = c->cls[cell * c->n_entries + e];
                w->rclosed[node] = mx <= q;
            }
            w->stats[0]++;
            if (found) {
                w->hit[node] = 1;
                for (int k = 0; k < 3; ++k) w->hitval[3 * node + k] = (double)c->rgb[3 * slot + k];
                w->stats[1]++;
                n_hit++;
            } else {
                w->stats[2]++;
            }
        }
        if (B->probe_key) B->probe_key[probe] = key;
        if (B->probe_cell) B->probe_cell[probe] = cell;
        if (B->probe_h2) B->probe_h2[probe] = h2;
        if (B->probe_hit) B->probe_hit[probe] = (uint8_t)found;
        probe++;
    }
    /* Needed set: the output is needed; a needed node that is not a hit root needs its
     * inputs (reverse storage order = reverse topological). */
    memset(w->needed, 0, M->n);
    w->needed[M->n - 1] = 1;
    for (int32_t j = (int32_t)M->n - 1; j >= 0; --j) {
        if (!w->needed[j] || w->hit[j]) continue;
        for (int k = 0; k < 4; ++k)
            if (M->nodes[j].in[k] >= 0) w->needed[M->nodes[j].in[k]] = 1;
    }
    /* Evaluation in storage order: hit roots take their cached value. */
    uint32_t n_eval = 0;
    double* val = w->val;
    for (uint32_t j = 0; j < M->n; ++j) {
        if (!w->needed[j]) continue;
        if (w->hit[j]) {
            for (int k = 0; k < 3; ++k) val[3 * j + k] = w->hitval[3 * j + k];
            continue;
        }
        const orc_node* nd = &M->nodes[j];
        orc_eval_node(nd, input_value(nd, 0, val), input_value(nd, 1, val), input_value(nd, 2, val), sp,
                      &val[3 * j]);
        n_eval++;
        if (!c->off && M->is_root[j] && w->rclosed[j]) {
            w->stats[3]++;
            w->stats[6]++;
        } else if (!c->off && M->is_root[j]) {
            /* A missed root that was evaluated becomes an insert candidate carrying its
             * own value rounded to FP32 (Sec. 3). */
            if (w->n_cand == w->cand_cap) {
                w->cand_cap *= 2;
                w->cand = (orc_candidate*)realloc(w->cand, w->cand_cap * sizeof(orc_candidate));
            }
            orc_candidate* cd = &w->cand[w->n_cand++];
            cd->cell = w->rcell[j];
            cd->h2 = w->rh2[j];
            cd->vis = B->vis ? B->vis[i] : 0;
            for (int k = 0; k < 3; ++k) cd->rgb[k] = (float)val[3 * j + k];
        }
    }
    w->stats[7] += n_eval;
    for (int k = 0; k < 3; ++k) B->rgb[(size_t)k * n + i] = val[3 * (M->n - 1) + k];
    if (B->hits) B->hits[i] = (uint16_t)n_hit;
    if (B->evaluated) B->evaluated[i] = n_eval;
}

/* Points per range of the all-core form. */
#define ORC_CHUNK 2048u

int orc_run_batch(orc_cache* c, uint64_t n, const float* u, const float* v,
                  const uint32_t* mat, const float* px, const float* py, const float* pz,
                  const float* nx, const float* ny, const float* nz, double* rgb,
                  uint16_t* hits, uint32_t* evaluated, uint64_t* probe_key,
                  uint64_t* probe_cell, uint32_t* probe_h2, uint8_t* probe_hit,
                  const float* g1u, const float* g1v, const float* g2u, const float* g2v,
                  const uint8_t* vis) {
    const orc_batch B = {n, u, v, mat, px, py, pz, nx, ny, nz, rgb, hits, evaluated, probe_key, probe_cell,
                         probe_h2, probe_hit, g1u, g1v, g2u, g2v, vis};
    uint32_t max_n = 1;
    for (uint32_t m = 0; m < c->n_mats; ++m)
        if (c->mats[m].n > max_n) max_n = c->mats[m].n;
    int status = ORC_OK;
    if (c->threads <= 1 || c->alg1) {
        /* one point after another */
        orc_work w;
        work_init(&w, max_n);
        uint64_t probe = 0;
        for (uint64_t i = 0; i < n; ++i) {
            process_point(c, &B, i, probe, &w);
            if (mat[i] < c->n_mats && !c->off) probe += c->mats[mat[i]].n_roots;
            if (c->alg1) {
                /* the paper's concurrent update, serialised one shading point at a time:
                 * the point's values are in the table before the next point looks up */
                for (int k = 0; k < ORC_NSTATS; ++k) c->stats[k] += w.stats[k];
                memset(w.stats, 0, sizeof(w.stats));
                c->stats[3] += w.n_cand;
                insert_candidates(c, w.cand, w.n_cand);
                w.n_cand = 0;
            }
        }
        for (int k = 0; k < ORC_NSTATS; ++k) c->stats[k] += w.stats[k];
        status = w.status;
        /* Phase I: candidates were produced in ascending (point index, node ID) order;
         * insert them one at a time in that order (Alg. 1 serialised: the CAS on an
         * empty entry always succeeds; the first value is kept). */
        c->stats[3] += w.n_cand;
        insert_candidates(c, w.cand, w.n_cand);
        work_free(&w);
    } else {
        /* All cores: ranges of points evaluated in parallel against the same snapshot of
         * the table (no point of phase L writes it), then every range's candidates in
         * range order, i.e. ascending (point index, node ID), inserted one at a time. */
        const uint64_t n_chunks = (n + ORC_CHUNK - 1) / ORC_CHUNK;
        uint64_t* probe0 = (uint64_t*)malloc((n_chunks + 1) * sizeof(uint64_t));
        probe0[0] = 0;
        for (uint64_t ch = 0; ch < n_chunks; ++ch) {
            uint64_t p = probe0[ch];
            for (uint64_t i = ch * ORC_CHUNK; i < n && i < (ch + 1) * ORC_CHUNK; ++i)
                if (mat[i] < c->n_mats && !c->off) p += c->mats[mat[i]].n_roots;
            probe0[ch + 1] = p;
        }
        orc_work* works = (orc_work*)malloc((n_chunks ? n_chunks : 1) * sizeof(orc_work));
#pragma omp parallel for schedule(dynamic, 1) num_threads(c->threads)
        for (int64_t ch = 0; ch < (int64_t)n_chunks; ++ch) {
            orc_work* w = &works[ch];
            work_init(w, max_n);
            uint64_t probe = probe0[ch];
            for (uint64_t i = (uint64_t)ch * ORC_CHUNK; i < n && i < ((uint64_t)ch + 1) * ORC_CHUNK; ++i) {
                process_point(c, &B, i, probe, w);
                if (mat[i] < c->n_mats && !c->off) probe += c->mats[mat[i]].n_roots;
            }
        }
        for (uint64_t ch = 0; ch < n_chunks; ++ch) {
            for (int k = 0; k < ORC_NSTATS; ++k) c->stats[k] += works[ch].stats[k];
            if (works[ch].status != ORC_OK) status = works[ch].status;
        }
        for (uint64_t ch = 0; ch < n_chunks; ++ch) {
            c->stats[3] += works[ch].n_cand;
            insert_candidates(c, works[ch].cand, works[ch].n_cand);
            work_free(&works[ch]);
        }
        free(works);
        free(probe0);
    }
    c->stats[8]++;
    return status;
}

void orc_cache_table(const orc_cache* c, uint32_t* h2, float* rgb) {
    size_t slots = c->off ? 0 : (size_t)c->n_cells * c->n_entries;
    if (slots) {
        memcpy(h2, c->h2, slots * sizeof(uint32_t));
        memcpy(rgb, c->rgb, 3 * slots * sizeof(float));
    }
}

void orc_cache_classes(const orc_cache* c, uint8_t* cls) {
    size_t slots = c->off ? 0 : (size_t)c->n_cells * c->n_entries;
    if (slots) memcpy(cls, c->cls, slots);
}

void orc_cache_stats(const orc_cache* c, uint64_t out[ORC_NSTATS]) {
    memcpy(out, c->stats, sizeof(c->stats));
}
