/*
 * Oracle fixed-accuracy block codec -- TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The paper compresses every checkpoint with ZFP in fixed-accuracy mode: the
 * caller fixes an absolute error tolerance atol and every decompressed value
 * stays within it (Sec. 1.4; Sec. 4.2 and the appendix figure on direct
 * compression report L_inf below atol).  The paper does not describe ZFP's
 * internals, so this project defines its own ZFP-style format from the
 * published structure of that method (4x4x4 blocks, a common block exponent,
 * a decorrelating transform, negabinary coefficients, embedded bit-plane
 * coding).  The steps below are written in that order, one function each,
 * plainly and without any blocking or fusion.
 *
 * Format constants:
 *   S = 25   fraction bits of the block-floating-point integers
 *   G = 11   guard planes: planes coded = emax - minexp + G (clamped 0..32)
 *   planes in {30, 31} are raised to 32 (lossless coefficient coding), so
 *   that every lossy block drops at least 3 planes; with this transform the
 *   worst-case error then stays below 2^minexp <= atol (pinned by the
 *   bound tests, which recompute the inverse-transform gain).
 *
 * Stream layout (little endian):
 *   [0,64)    header: magic, version, nx, ny, nz, minexp, nblocks,
 *             chunk size (32 blocks), nchunks, payload words, total bytes,
 *             format parameters
 *   then      nchunks x u64   word offset of each chunk in the payload
 *   then      nblocks x u16   bit length of each block (padded to 8 bytes)
 *   then      payload: u64 words; the blocks of one chunk are concatenated
 *             LSB-first, and every chunk starts on a fresh word.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ZO_S 25
#define ZO_G 11
#define ZO_CHUNK 32
#define ZO_MAXBITS (9 + 32 * 64 + 64)
#define ZO_MAGIC 0x315A4346u /* "FCZ1" */
#define ZO_VERSION 1u
#define ZO_NBMASK 0xAAAAAAAAu

/* ---- bit I/O ------------------------------------------------------------ */

typedef struct {
  uint64_t* w;
  long nwords;
  long pos; /* bit position */
} zo_writer;

static int zo_put_bit(zo_writer* bw, unsigned bit) {
  long word = bw->pos >> 6;
  if (word >= bw->nwords) return ORACLE_ERR_CAPACITY;
  if (bit) bw->w[word] |= (uint64_t)1 << (bw->pos & 63);
  bw->pos++;
  return 0;
}

static int zo_put_bits(zo_writer* bw, uint64_t value, int n) {
  for (int i = 0; i < n; i++) {
    int s = zo_put_bit(bw, (unsigned)((value >> i) & 1u));
    if (s) return s;
  }
  return 0;
}

typedef struct {
  const uint64_t* w;
  long nbits;
  long pos;
} zo_reader;

static int zo_get_bit(zo_reader* br, unsigned* bit) {
  if (br->pos >= br->nbits) return ORACLE_ERR_CORRUPT;
  *bit = (unsigned)((br->w[br->pos >> 6] >> (br->pos & 63)) & 1u);
  br->pos++;
  return 0;
}

static int zo_get_bits(zo_reader* br, int n, uint64_t* value) {
  uint64_t v = 0;
  for (int i = 0; i < n; i++) {
    unsigned b;
    int s = zo_get_bit(br, &b);
    if (s) return s;
    v |= (uint64_t)b << i;
  }
  *value = v;
  return 0;
}

/* ---- step 1: tolerance -> minimum exponent ------------------------------ */

/* minexp = floor(log2(atol)), exactly: atol = f 2^e with f in [0.5, 1). */
int oracle_zfp_minexp(double atol) {
  int e;
  frexp(atol, &e);
  return e - 1;
}

/* ---- step 2: block exponent and coded-plane count ------------------------ */

static int zo_planes(int emax, int minexp) {
  int p = emax - minexp + ZO_G;
  if (p < 0) p = 0;
  if (p > 32) p = 32;
  if (p == 30 || p == 31) p = 32;
  return p;
}

/* Largest frexp exponent over the block (x = f 2^e, f in [0.5,1)), clamped
 * below at -127 so that emax+127 fits 8 bits (a larger emax still bounds
 * every |x|); sets *planes = 0 for an all-zero block.  Then step 3, the
 * block-floating-point integers. */
int oracle_zfp_block_quantise(const float v[64], int minexp, int32_t q[64],
                              int* emax_out, int* planes) {
  int have = 0, em = -100000;
  for (int i = 0; i < 64; i++) {
    if (!isfinite(v[i])) return ORACLE_ERR_NONFINITE;
    if (v[i] != 0.0f) {
      int e;
      frexp((double)v[i], &e);
      if (!have || e > em) em = e;
      have = 1;
    }
  }
  if (!have) {
    *emax_out = 0;
    *planes = 0;
    for (int i = 0; i < 64; i++) q[i] = 0;
    return 0;
  }
  if (em < -127) em = -127;
  *emax_out = em;
  *planes = zo_planes(em, minexp);
  /* step 3: block floating point, q = trunc(x 2^(S-emax)); exact in double */
  for (int i = 0; i < 64; i++) q[i] = (int32_t)trunc(ldexp((double)v[i], ZO_S - em));
  return 0;
}

/* ---- step 4: decorrelating integer lifting transform --------------------- */

/* Floor division by two of a signed integer (an arithmetic shift). */
static int32_t zo_half(int32_t a) { return (int32_t)floor((double)a / 2.0); }

/* Four samples x0..x3 -> (S, D, d0, d1): pair differences and floor means,
 * the same on the two means, then the linear trend (D/2) removed from both
 * fine differences.  Every step adds a function of other entries, so the
 * inverse below runs the same steps backwards with the signs flipped. */
void oracle_zfp_fwd_lift4(int32_t* p, int s) {
  int32_t x0 = p[0], x1 = p[s], x2 = p[2 * s], x3 = p[3 * s];
  int32_t d0 = x1 - x0;
  int32_t s0 = x0 + zo_half(d0);
  int32_t d1 = x3 - x2;
  int32_t s1 = x2 + zo_half(d1);
  int32_t D = s1 - s0;
  int32_t S = s0 + zo_half(D);
  d0 = d0 - zo_half(D);
  d1 = d1 - zo_half(D);
  p[0] = S;
  p[s] = D;
  p[2 * s] = d0;
  p[3 * s] = d1;
}

void oracle_zfp_inv_lift4(int32_t* p, int s) {
  int32_t S = p[0], D = p[s], d0 = p[2 * s], d1 = p[3 * s];
  d1 = d1 + zo_half(D);
  d0 = d0 + zo_half(D);
  int32_t s0 = S - zo_half(D);
  int32_t s1 = D + s0;
  int32_t x2 = s1 - zo_half(d1);
  int32_t x3 = d1 + x2;
  int32_t x0 = s0 - zo_half(d0);
  int32_t x1 = d0 + x0;
  p[0] = x0;
  p[s] = x1;
  p[2 * s] = x2;
  p[3 * s] = x3;
}

/* Along x (16 lines), then y, then z. */
void oracle_zfp_fwd_xform(int32_t q[64]) {
  for (int k = 0; k < 4; k++)
    for (int j = 0; j < 4; j++) oracle_zfp_fwd_lift4(q + 4 * j + 16 * k, 1);
  for (int k = 0; k < 4; k++)
    for (int i = 0; i < 4; i++) oracle_zfp_fwd_lift4(q + i + 16 * k, 4);
  for (int j = 0; j < 4; j++)
    for (int i = 0; i < 4; i++) oracle_zfp_fwd_lift4(q + i + 4 * j, 16);
}

/* Along z, then y, then x. */
void oracle_zfp_inv_xform(int32_t q[64]) {
  for (int j = 0; j < 4; j++)
    for (int i = 0; i < 4; i++) oracle_zfp_inv_lift4(q + i + 4 * j, 16);
  for (int k = 0; k < 4; k++)
    for (int i = 0; i < 4; i++) oracle_zfp_inv_lift4(q + i + 16 * k, 4);
  for (int k = 0; k < 4; k++)
    for (int j = 0; j < 4; j++) oracle_zfp_inv_lift4(q + 4 * j + 16 * k, 1);
}

/* ---- step 5: coefficient order ------------------------------------------ */

/* Ascending total sequency i+j+k; ties by the x-fastest index.  A plain
 * selection over the 64 keys. */
void oracle_zfp_perm(int perm[64]) {
  int used[64] = {0};
  for (int p = 0; p < 64; p++) {
    int best = -1, bestkey = 1 << 30;
    for (int idx = 0; idx < 64; idx++) {
      if (used[idx]) continue;
      int i = idx & 3, j = (idx >> 2) & 3, k = idx >> 4;
      int key = (i + j + k) * 64 + idx;
      if (key < bestkey) {
        bestkey = key;
        best = idx;
      }
    }
    used[best] = 1;
    perm[p] = best;
  }
}

/* ---- step 6: negabinary ------------------------------------------------- */

static uint32_t zo_to_negabinary(int32_t c) {
  return ((uint32_t)c + ZO_NBMASK) ^ ZO_NBMASK;
}
static int32_t zo_from_negabinary(uint32_t u) {
  return (int32_t)((u ^ ZO_NBMASK) - ZO_NBMASK);
}

/* ---- step 7: embedded bit-plane coding of one block --------------------- */

static int zo_encode_block(const float v[64], int minexp, zo_writer* bw) {
  int32_t q[64];
  int emax, planes;
  int s = oracle_zfp_block_quantise(v, minexp, q, &emax, &planes);
  if (s) return s;
  if (planes == 0) return zo_put_bit(bw, 0);
  if ((s = zo_put_bit(bw, 1))) return s;
  if ((s = zo_put_bits(bw, (uint64_t)(emax + 127), 8))) return s;
  oracle_zfp_fwd_xform(q);
  int perm[64];
  oracle_zfp_perm(perm);
  uint32_t u[64];
  for (int p = 0; p < 64; p++) u[p] = zo_to_negabinary(q[perm[p]]);
  int n = 0; /* coefficients already significant */
  for (int b = 31; b >= 32 - planes; b--) {
    for (int i = 0; i < n; i++)
      if ((s = zo_put_bit(bw, (u[i] >> b) & 1u))) return s;
    while (n < 64) {
      unsigned any = 0;
      for (int i = n; i < 64; i++) any |= (u[i] >> b) & 1u;
      if ((s = zo_put_bit(bw, any))) return s;
      if (!any) break;
      unsigned bit;
      do {
        bit = (u[n] >> b) & 1u;
        if ((s = zo_put_bit(bw, bit))) return s;
        n++;
      } while (!bit);
    }
  }
  return 0;
}

static int zo_decode_block(zo_reader* br, int minexp, float v[64]) {
  unsigned flag;
  int s = zo_get_bit(br, &flag);
  if (s) return s;
  if (!flag) {
    for (int i = 0; i < 64; i++) v[i] = 0.0f;
    return 0;
  }
  uint64_t eb;
  if ((s = zo_get_bits(br, 8, &eb))) return s;
  int emax = (int)eb - 127;
  int planes = zo_planes(emax, minexp);
  if (planes == 0) return ORACLE_ERR_CORRUPT;
  uint32_t u[64] = {0};
  int n = 0;
  for (int b = 31; b >= 32 - planes; b--) {
    for (int i = 0; i < n; i++) {
      unsigned bit;
      if ((s = zo_get_bit(br, &bit))) return s;
      u[i] |= (uint32_t)bit << b;
    }
    while (n < 64) {
      unsigned any;
      if ((s = zo_get_bit(br, &any))) return s;
      if (!any) break;
      unsigned bit;
      do {
        if (n >= 64) return ORACLE_ERR_CORRUPT;
        if ((s = zo_get_bit(br, &bit))) return s;
        u[n] |= (uint32_t)bit << b;
        n++;
      } while (!bit);
    }
  }
  int perm[64];
  oracle_zfp_perm(perm);
  int32_t q[64];
  for (int p = 0; p < 64; p++) q[perm[p]] = zo_from_negabinary(u[p]);
  oracle_zfp_inv_xform(q);
  /* back to FP32: one rounding of the exact product q 2^(emax-S) */
  for (int i = 0; i < 64; i++) v[i] = (float)ldexp((double)q[i], emax - ZO_S);
  return 0;
}

int oracle_zfp_encode_block(const float v[64], int minexp, uint64_t* bits, int nwords) {
  memset(bits, 0, sizeof(uint64_t) * (size_t)nwords);
  zo_writer bw = {bits, nwords, 0};
  int s = zo_encode_block(v, minexp, &bw);
  return s ? s : (int)bw.pos;
}

int oracle_zfp_decode_block(const uint64_t* bits, int nbits, int minexp, float v[64]) {
  zo_reader br = {bits, nbits, 0};
  int s = zo_decode_block(&br, minexp, v);
  return s ? s : (int)br.pos;
}

/* ---- whole-field stream ------------------------------------------------- */

static long zo_ceil_div(long a, long b) { return (a + b - 1) / b; }

typedef struct {
  long nbx, nby, nbz, nblocks, nchunks;
  size_t chunk_table, length_table, payload; /* byte offsets */
} zo_layout;

static void zo_make_layout(int nx, int ny, int nz, zo_layout* L) {
  L->nbx = zo_ceil_div(nx, 4);
  L->nby = zo_ceil_div(ny, 4);
  L->nbz = zo_ceil_div(nz, 4);
  L->nblocks = L->nbx * L->nby * L->nbz;
  L->nchunks = zo_ceil_div(L->nblocks, ZO_CHUNK);
  L->chunk_table = 64;
  L->length_table = L->chunk_table + 8 * (size_t)L->nchunks;
  L->payload = L->length_table + (size_t)zo_ceil_div(2 * L->nblocks, 8) * 8;
}

size_t oracle_zfp_max_bytes(int nx, int ny, int nz) {
  if (nx <= 0 || ny <= 0 || nz <= 0) return 0;
  zo_layout L;
  zo_make_layout(nx, ny, nz, &L);
  size_t words = 0;
  for (long c = 0; c < L.nchunks; c++) {
    long nb = L.nblocks - c * ZO_CHUNK;
    if (nb > ZO_CHUNK) nb = ZO_CHUNK;
    words += (size_t)zo_ceil_div(nb * ZO_MAXBITS, 64);
  }
  return L.payload + 8 * words;
}

/* Gather block b (x fastest) with edge replication for partial blocks. */
static void zo_gather(const float* in, int nx, int ny, int nz, const zo_layout* L,
                      long b, float v[64]) {
  long bx = b % L->nbx, by = (b / L->nbx) % L->nby, bz = b / (L->nbx * L->nby);
  for (int k = 0; k < 4; k++)
    for (int j = 0; j < 4; j++)
      for (int i = 0; i < 4; i++) {
        long x = 4 * bx + i, y = 4 * by + j, z = 4 * bz + k;
        if (x > nx - 1) x = nx - 1;
        if (y > ny - 1) y = ny - 1;
        if (z > nz - 1) z = nz - 1;
        v[i + 4 * j + 16 * k] = in[x + (long)nx * (y + (long)ny * z)];
      }
}

static void zo_scatter(float* out, int nx, int ny, int nz, const zo_layout* L, long b,
                       const float v[64]) {
  long bx = b % L->nbx, by = (b / L->nbx) % L->nby, bz = b / (L->nbx * L->nby);
  for (int k = 0; k < 4; k++)
    for (int j = 0; j < 4; j++)
      for (int i = 0; i < 4; i++) {
        long x = 4 * bx + i, y = 4 * by + j, z = 4 * bz + k;
        if (x < nx && y < ny && z < nz) out[x + (long)nx * (y + (long)ny * z)] = v[i + 4 * j + 16 * k];
      }
}

static void zo_put_u32(uint8_t* p, uint32_t v) { memcpy(p, &v, 4); }
static void zo_put_u64(uint8_t* p, uint64_t v) { memcpy(p, &v, 8); }
static uint32_t zo_get_u32(const uint8_t* p) { uint32_t v; memcpy(&v, p, 4); return v; }
static uint64_t zo_get_u64(const uint8_t* p) { uint64_t v; memcpy(&v, p, 8); return v; }

int oracle_zfp_compress(const float* in, int nx, int ny, int nz, double atol,
                        uint8_t* out, size_t cap, size_t* out_bytes) {
  if (!in || nx <= 0 || ny <= 0 || nz <= 0 || !(atol > 0.0) || !isfinite(atol) || !out_bytes)
    return ORACLE_ERR_ARG;
  int minexp = oracle_zfp_minexp(atol);
  zo_layout L;
  zo_make_layout(nx, ny, nz, &L);
  uint64_t* chunk_off = (uint64_t*)calloc((size_t)L.nchunks, 8);
  uint16_t* lengths = (uint16_t*)calloc((size_t)L.nblocks, 2);
  size_t maxwords = (oracle_zfp_max_bytes(nx, ny, nz) - L.payload) / 8;
  uint64_t* payload = (uint64_t*)calloc(maxwords, 8);
  if (!chunk_off || !lengths || !payload) {
    free(chunk_off); free(lengths); free(payload);
    return ORACLE_ERR_NOMEM;
  }
  int status = 0;
  long word = 0;
  for (long c = 0; c < L.nchunks && !status; c++) {
    chunk_off[c] = (uint64_t)word;
    zo_writer bw = {payload + word, (long)maxwords - word, 0};
    for (long b = c * ZO_CHUNK; b < L.nblocks && b < (c + 1) * ZO_CHUNK; b++) {
      float v[64];
      zo_gather(in, nx, ny, nz, &L, b, v);
      long before = bw.pos;
      status = zo_encode_block(v, minexp, &bw);
      if (status) break;
      lengths[b] = (uint16_t)(bw.pos - before);
    }
    word += zo_ceil_div(bw.pos, 64);
  }
  size_t total = L.payload + 8 * (size_t)word;
  if (!status) {
    *out_bytes = total;
    if (total > cap || !out) {
      status = ORACLE_ERR_CAPACITY;
    } else {
      memset(out, 0, L.payload);
      zo_put_u32(out + 0, ZO_MAGIC);
      zo_put_u32(out + 4, ZO_VERSION);
      zo_put_u32(out + 8, (uint32_t)nx);
      zo_put_u32(out + 12, (uint32_t)ny);
      zo_put_u32(out + 16, (uint32_t)nz);
      zo_put_u32(out + 20, (uint32_t)minexp);
      zo_put_u64(out + 24, (uint64_t)L.nblocks);
      zo_put_u32(out + 32, ZO_CHUNK);
      zo_put_u32(out + 36, (uint32_t)L.nchunks);
      zo_put_u64(out + 40, (uint64_t)word);
      zo_put_u64(out + 48, (uint64_t)total);
      zo_put_u32(out + 56, (uint32_t)(ZO_S | (ZO_G << 8)));
      zo_put_u32(out + 60, 0u);
      for (long c = 0; c < L.nchunks; c++) zo_put_u64(out + L.chunk_table + 8 * c, chunk_off[c]);
      for (long b = 0; b < L.nblocks; b++) memcpy(out + L.length_table + 2 * b, &lengths[b], 2);
      for (long w = 0; w < word; w++) zo_put_u64(out + L.payload + 8 * w, payload[w]);
    }
  }
  free(chunk_off);
  free(lengths);
  free(payload);
  return status;
}

int oracle_zfp_decompress(const uint8_t* in, size_t in_bytes, float* out, int nx, int ny, int nz) {
  if (!in || !out || nx <= 0 || ny <= 0 || nz <= 0) return ORACLE_ERR_ARG;
  if (in_bytes < 64) return ORACLE_ERR_CORRUPT;
  zo_layout L;
  zo_make_layout(nx, ny, nz, &L);
  if (zo_get_u32(in) != ZO_MAGIC || zo_get_u32(in + 4) != ZO_VERSION) return ORACLE_ERR_CORRUPT;
  if ((int)zo_get_u32(in + 8) != nx || (int)zo_get_u32(in + 12) != ny ||
      (int)zo_get_u32(in + 16) != nz)
    return ORACLE_ERR_ARG;
  int minexp = (int32_t)zo_get_u32(in + 20);
  uint64_t words = zo_get_u64(in + 40);
  if (zo_get_u64(in + 24) != (uint64_t)L.nblocks || zo_get_u32(in + 32) != ZO_CHUNK ||
      zo_get_u32(in + 36) != (uint32_t)L.nchunks || zo_get_u32(in + 56) != (uint32_t)(ZO_S | (ZO_G << 8)))
    return ORACLE_ERR_CORRUPT;
  if (L.payload > in_bytes || words > (in_bytes - L.payload) / 8) return ORACLE_ERR_CORRUPT;
  uint64_t* payload = (uint64_t*)malloc((size_t)(words ? words : 1) * 8);
  if (!payload) return ORACLE_ERR_NOMEM;
  for (uint64_t w = 0; w < words; w++) payload[w] = zo_get_u64(in + L.payload + 8 * w);
  int status = 0;
  for (long c = 0; c < L.nchunks && !status; c++) {
    uint64_t start = zo_get_u64(in + L.chunk_table + 8 * c);
    uint64_t end = (c + 1 < L.nchunks) ? zo_get_u64(in + L.chunk_table + 8 * (c + 1)) : words;
    if (start > end || end > words) { status = ORACLE_ERR_CORRUPT; break; }
    long pos = 0;
    for (long b = c * ZO_CHUNK; b < L.nblocks && b < (c + 1) * ZO_CHUNK; b++) {
      uint16_t len;
      memcpy(&len, in + L.length_table + 2 * b, 2);
      /* the reader may not run past this block's recorded length */
      long limit = pos + len;
      if (limit > (long)(64 * (end - start))) { status = ORACLE_ERR_CORRUPT; break; }
      zo_reader br = {payload + start, limit, pos};
      float v[64];
      status = zo_decode_block(&br, minexp, v);
      if (status) break;
      if (br.pos != limit) { status = ORACLE_ERR_CORRUPT; break; }
      zo_scatter(out, nx, ny, nz, &L, b, v);
      pos = limit;
    }
  }
  free(payload);
  return status;
}
