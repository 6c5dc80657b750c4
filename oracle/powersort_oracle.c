/*
 * Powersort oracle: a plain, slow, single-threaded CPU statement of what the
 * paper "Virtual-Memory Powersort" (Moltmann, Nakajima, Wild) computes.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path may call this code;
 * only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark load it.  It shares no source with the CUDA implementation.
 *
 * Contents (each follows the passage named beside it):
 *   oracle_minrun        minimum run length rule, Sec. 5 "Algorithm variants"
 *   oracle_power         Power(n, a, b) by its definition, Sec. 2 Theorem
 *   oracle_stable_sort   the plain definition of the result: the unique stable
 *                        order (Sec. 1: equal elements keep their input order)
 *   oracle_powersort     Algorithm 1 ("Abstract Powersort") executed literally
 *                        with Pingpong storage (Sec. 3) and StandardMerge
 *                        (Algorithm 2, right), recording runs, powers, the
 *                        merges in execution order, the merge cost M
 *                        (Sec. 2 Definition), the stack height and the
 *                        comparison / move counters of Sec. 5-6.
 *   oracle_powersort_vm  Algorithm 1 with the virtual-memory buffers of Sec. 4:
 *                        runs as page lists, a free list, PageMerge
 *                        (Algorithm 2, left) and the final page-permuting Copy;
 *                        it reports the peak number of pages in use.
 *   oracle_powersort_ex, oracle_powersort_vm_ex
 *                        the same with options; ORACLE_DESCENDING_RUNS takes
 *                        the variant of Sec. 5 "Algorithm variants" that also
 *                        accepts decreasing runs (reversed in place);
 *                        ORACLE_KEY_I32 / ORACLE_KEY_F32 read the 32-bit keys
 *                        as two's-complement integers / IEEE-754 binary32
 *                        values ordered by the standard's totalOrder
 *   oracle_stable_sort_ex the stable-sort definition under those key orders
 *   oracle_stable_rank_ex one output of that definition: the stable position
 *                        of a single element
 *   oracle_powersort_keys64
 *                        64-bit keys (unsigned, two's complement, or IEEE 754
 *                        binary64 under totalOrder): Algorithm 1 on indices,
 *                        comparing the keys by those definitions
 *   oracle_powersort_records, oracle_stable_sort_records
 *                        the same for records of `words` 32-bit words ordered
 *                        lexicographically (the paper's blob types, Sec. 5
 *                        "Input data types"): the keys are record indices
 *                        compared through the rows
 *
 * Readings taken where the paper is silent:
 *   - indices are 0-based and half open: a = [i, j), b = [j, k);
 *   - the final loop of Algorithm 1 pops the stack after every merge;
 *   - minrun for n < 64 is n (the halving loop never runs);
 *   - a forced run ends at min(s + minrun, n) and is not re-scanned after the
 *     insertion sort; a natural run at least minrun long is kept whole;
 *   - decreasing runs (variant): a run whose first two elements are in
 *     strictly decreasing order continues while the order stays strictly
 *     decreasing and is then reversed (strictness keeps equal elements in
 *     input order, so the sort stays stable); a shorter one than minrun is
 *     extended and insertion-sorted like any other forced run.
 * Parity is pinned for every function here (no "parity unpinned" entries).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    uint64_t n;
    uint64_t runs;               /* number of runs found by ExtractRun        */
    uint64_t merges;             /* number of MergeBuffers calls              */
    uint64_t merge_cost;         /* M: sum of the lengths of all merge inputs */
    uint64_t comparisons;        /* key comparisons: scans + merges + inserts */
    uint64_t merge_comparisons;  /* comparisons made inside merges only       */
    uint64_t scan_comparisons;   /* comparisons made by the run scans         */
    uint64_t insert_comparisons; /* comparisons made by insertion sort        */
    uint64_t moves;              /* element moves of merges + buffer copies   */
    uint64_t insert_moves;       /* element moves made by insertion sort      */
    uint64_t peak_pages;         /* VM storage: peak pages in use (else 0)    */
    uint64_t pool_pages;         /* VM storage: pages taken beyond the input  */
    uint32_t minrun;
    uint32_t max_stack;          /* largest stack height seen                 */
    uint32_t max_power;          /* largest boundary power                    */
    uint32_t page_size;          /* VM storage: P (else 0)                    */
    uint64_t reversed_runs;      /* decreasing runs found and reversed        */
    uint64_t reverse_moves;      /* element moves made by the reversals       */
} oracle_stats;

/* options of oracle_powersort_ex / oracle_powersort_vm_ex / oracle_stable_sort_ex */
#define ORACLE_DESCENDING_RUNS 1u
#define ORACLE_KEY_I32 2u
#define ORACLE_KEY_F32 4u
#define ORACLE_RECORDS 8u
#define ORACLE_KEYS64 16u   /* with ORACLE_KEY_I32 / ORACLE_KEY_F32: int64 / binary64 */

/* The 64-bit keys of the running call (ORACLE_KEYS64). */
static const uint64_t* g_keys64;

/* The records of the running call (ORACLE_RECORDS): row i is
 * g_rec[i * g_rec_words .. (i + 1) * g_rec_words). */
static const uint32_t* g_rec;
static uint32_t g_rec_words;

/* The key order of the running call (the oracle is single-threaded). */
static uint32_t g_key_order;

/* key_gt(a, b): key a sorts strictly after key b.
 *   default        unsigned 32-bit integers;
 *   ORACLE_KEY_I32 two's-complement 32-bit integers;
 *   ORACLE_KEY_F32 IEEE 754 binary32 totalOrder (IEEE 754-2008 Sec. 5.10):
 *                  negative values (sign bit set) precede positive ones;
 *                  among positives a larger bit pattern (exponent, then
 *                  fraction, then NaN payload) is larger; among negatives the
 *                  order of the magnitudes is reversed.  So -NaN < -inf <
 *                  ... < -0 < +0 < ... < +inf < +NaN. */
static int key_gt(uint32_t a, uint32_t b)
{
    if (g_key_order & ORACLE_KEYS64) {
        /* indices of 64-bit keys; the same three orders at 64 bits */
        const uint64_t x = g_keys64[a], y = g_keys64[b];
        if (g_key_order & ORACLE_KEY_I32) return (int64_t)x > (int64_t)y;
        if (g_key_order & ORACLE_KEY_F32) {
            const int nx = (int)(x >> 63), ny = (int)(y >> 63);
            if (nx != ny) return ny;
            const uint64_t mx = x & 0x7fffffffffffffffull, my = y & 0x7fffffffffffffffull;
            return nx ? mx < my : mx > my;
        }
        return x > y;
    }
    if (g_key_order & ORACLE_RECORDS) {
        /* lexicographic: the first differing word (as unsigned) decides */
        const uint32_t* ra = g_rec + (uint64_t)a * g_rec_words;
        const uint32_t* rb = g_rec + (uint64_t)b * g_rec_words;
        for (uint32_t w = 0; w < g_rec_words; ++w)
            if (ra[w] != rb[w]) return ra[w] > rb[w];
        return 0;
    }
    if (g_key_order & ORACLE_KEY_I32) return (int32_t)a > (int32_t)b;
    if (g_key_order & ORACLE_KEY_F32) {
        const int na = (int)(a >> 31), nb = (int)(b >> 31);
        if (na != nb) return nb;                        /* a positive, b negative */
        const uint32_t ma = a & 0x7fffffffu, mb = b & 0x7fffffffu;
        return na ? ma < mb : ma > mb;
    }
    return a > b;
}

/* Sec. 5, "Algorithm variants": start from l = n and halve (rounding up)
 * until l < 64.  When n < 64 the loop body never runs and minrun = n. */
uint32_t oracle_minrun(uint64_t n)
{
    uint64_t l = n;
    while (l >= 64) l = (l + 1) / 2;
    return (uint32_t)l;
}

/* Sec. 2 Theorem: Power(n, a, b) for a = [i, j), b = [j, k) is the smallest
 * integer p such that some integer c has (i+j)/(2n) < c / 2^p <= (j+k)/(2n).
 * Such a c exists exactly when floor((j+k) 2^p / (2n)) > floor((i+j) 2^p / (2n))
 * (c = the larger floor).  The search runs p = 0, 1, 2, ... in 128-bit
 * integers so no rounding can occur. */
uint32_t oracle_power(uint64_t n, uint64_t i, uint64_t j, uint64_t k)
{
    unsigned __int128 two_n = (unsigned __int128)2 * n;
    for (uint32_t p = 0; p < 100; ++p) {
        unsigned __int128 lo = (((unsigned __int128)(i + j)) << p) / two_n;
        unsigned __int128 hi = (((unsigned __int128)(j + k)) << p) / two_n;
        if (hi > lo) return p;
    }
    return 0xffffffffu; /* unreachable for i < j < k <= n */
}

/* ------------------------------------------------------------------------- */
/* The plain definition of the result: the unique stable sort.  Output rank r
 * holds the element whose (key, input index) pair is the r-th smallest.  The
 * library routine qsort orders the pairs; ties on the key are broken by the
 * input index, which is exactly what stability demands (Sec. 1). */
typedef struct { uint32_t key; uint32_t idx; } kv_pair;

static int cmp_pair(const void* x, const void* y)
{
    const kv_pair* a = (const kv_pair*)x;
    const kv_pair* b = (const kv_pair*)y;
    if (key_gt(a->key, b->key)) return 1;
    if (key_gt(b->key, a->key)) return -1;
    if (a->idx != b->idx) return a->idx < b->idx ? -1 : 1;
    return 0;
}

int oracle_stable_sort_ex(const uint32_t* keys, uint64_t n, uint32_t options, uint32_t* keys_out,
                          uint32_t* perm_out)
{
    g_key_order = options & (ORACLE_KEY_I32 | ORACLE_KEY_F32 | ORACLE_RECORDS | ORACLE_KEYS64);
    if (n == 0) return 0;
    kv_pair* v = (kv_pair*)malloc(n * sizeof(kv_pair));
    if (!v) return -1;
    for (uint64_t x = 0; x < n; ++x) { v[x].key = keys[x]; v[x].idx = (uint32_t)x; }
    qsort(v, n, sizeof(kv_pair), cmp_pair);
    for (uint64_t x = 0; x < n; ++x) {
        if (keys_out) keys_out[x] = v[x].key;
        if (perm_out) perm_out[x] = v[x].idx;
    }
    free(v);
    return 0;
}

int oracle_stable_sort(const uint32_t* keys, uint64_t n, uint32_t* keys_out, uint32_t* perm_out)
{
    return oracle_stable_sort_ex(keys, n, 0u, keys_out, perm_out);
}

/* One output of the same definition: the position that element i takes in
 * the stable order, i.e. the number of elements j that come before it (a
 * smaller key, or an equal key and j < i).  Lets a check of a very large sort
 * sample its outputs one by one in O(n) each. */
uint64_t oracle_stable_rank_ex(const uint32_t* keys, uint64_t n, uint32_t options, uint64_t i)
{
    g_key_order = options & (ORACLE_KEY_I32 | ORACLE_KEY_F32);
    uint64_t r = 0;
    for (uint64_t j = 0; j < n; ++j)
        r += key_gt(keys[i], keys[j]) || (j < i && !key_gt(keys[j], keys[i]));
    return r;
}

/* ------------------------------------------------------------------------- */
/* ExtractRun (Sec. 2 operation list; Sec. 3: "looks for the first pair of
 * adjacent elements in the wrong order") with the minimum-run-length rule of
 * Sec. 5: a run shorter than minrun is extended to min(s + minrun, n)
 * elements and sorted by (stable) insertion sort.  Returns the run end. */
static uint64_t extract_run(uint32_t* key, uint32_t* perm, uint64_t s, uint64_t n,
                            uint32_t minrun, uint32_t options, oracle_stats* st)
{
    uint64_t e = s + 1;
    int down = 0;
    if ((options & ORACLE_DESCENDING_RUNS) && e < n) {
        st->scan_comparisons++;
        down = key_gt(key[s], key[e]);
    }
    if (down) {
        /* strictly decreasing run: extend while a[e-1] > a[e], then reverse */
        ++e;
        while (e < n) {
            st->scan_comparisons++;
            if (!key_gt(key[e - 1], key[e])) break;
            ++e;
        }
        for (uint64_t x = s, y = e - 1; x < y; ++x, --y) {
            uint32_t tk = key[x], tp = perm[x];
            key[x] = key[y]; perm[x] = perm[y];
            key[y] = tk; perm[y] = tp;
            st->reverse_moves += 2;
        }
        st->reversed_runs++;
    } else {
        if (e < n && (options & ORACLE_DESCENDING_RUNS)) ++e;   /* pair (s, s+1) already compared */
        while (e < n) {
            st->scan_comparisons++;
            if (key_gt(key[e - 1], key[e])) break;   /* first descent: run ends here */
            ++e;
        }
    }
    if (e - s < minrun) {
        uint64_t end = s + minrun < n ? s + minrun : n;
        /* insertion sort of key[s, end); key[s, e) is already sorted */
        for (uint64_t x = e; x < end; ++x) {
            uint32_t v = key[x], pv = perm[x];
            uint64_t y = x;
            while (y > s) {
                st->insert_comparisons++;
                if (!key_gt(key[y - 1], v)) break; /* strict: equal keys stay put */
                key[y] = key[y - 1];
                perm[y] = perm[y - 1];
                st->insert_moves++;
                --y;
            }
            if (y != x) { key[y] = v; perm[y] = pv; st->insert_moves++; }
        }
        e = end;
    }
    return e;
}

/* StandardMerge (Algorithm 2, right) in Pingpong form (Sec. 3): the stack run
 * lives in stackBuf[i, j), curr in input[j, k); the result goes to input[i, k)
 * left to right.  Ties take the left (stack) run: a[xa] <= b[xb].  When the
 * left run runs out, the rest of the right run is already in place. */
static void pingpong_merge(uint32_t* key, uint32_t* perm, const uint32_t* bkey,
                           const uint32_t* bperm, uint64_t i, uint64_t j, uint64_t k,
                           oracle_stats* st)
{
    uint64_t xa = i, xb = j, xr = i;
    while (xa < j && xb < k) {
        st->merge_comparisons++;
        if (!key_gt(bkey[xa], key[xb])) { key[xr] = bkey[xa]; perm[xr] = bperm[xa]; ++xa; }
        else                     { key[xr] = key[xb];  perm[xr] = perm[xb];  ++xb; }
        ++xr;
        st->moves++;
    }
    while (xa < j) { key[xr] = bkey[xa]; perm[xr] = bperm[xa]; ++xa; ++xr; st->moves++; }
    /* xb < k: input[xb, k) is already at input[xr, k) since xr == xb */
}

/* The last-pop variant of Sec. 3 (final paragraph): the same merge, but the
 * result goes to stackBuf[i, k) and is produced right to left, so the run
 * that is pushed next needs no copy.  Going right to left, ties take the
 * right run (b), which yields the same stable order.  When the right run runs
 * out first, the rest of the left run is already in place. */
static void pingpong_merge_to_stack(const uint32_t* key, const uint32_t* perm, uint32_t* bkey,
                                    uint32_t* bperm, uint64_t i, uint64_t j, uint64_t k,
                                    oracle_stats* st)
{
    uint64_t xa = j, xb = k, xr = k;     /* one past the next element to take */
    while (xa > i && xb > j) {
        st->merge_comparisons++;
        --xr;
        if (key_gt(bkey[xa - 1], key[xb - 1])) { bkey[xr] = bkey[xa - 1]; bperm[xr] = bperm[xa - 1]; --xa; }
        else                            { bkey[xr] = key[xb - 1];  bperm[xr] = perm[xb - 1];  --xb; }
        st->moves++;
    }
    while (xb > j) { --xr; --xb; bkey[xr] = key[xb]; bperm[xr] = perm[xb]; st->moves++; }
    /* xa > i: stackBuf[i, xa) is already in place since xr == xa */
}

/* Algorithm 1 ("Abstract Powersort") with Pingpong storage (Sec. 3).
 *   key[0, n), perm[0, n): in/out; perm is filled with 0..n-1 first.
 *   run_starts: receives the start of every run plus n (runs + 1 entries).
 *   powers:     powers[t] = Power of the boundary between run t and run t+1.
 *   merges:     (lo, mid, hi) triples in execution order.
 *   options:    ORACLE_DESCENDING_RUNS or 0.
 * Any output pointer may be NULL.  Returns 0, or -1 on allocation failure. */
int oracle_powersort_ex(uint32_t* key, uint32_t* perm, uint64_t n, uint32_t* run_starts,
                        uint8_t* powers, uint32_t* merges, uint32_t options, oracle_stats* st)
{
    memset(st, 0, sizeof(*st));
    g_key_order = options & (ORACLE_KEY_I32 | ORACLE_KEY_F32 | ORACLE_RECORDS | ORACLE_KEYS64);
    st->n = n;
    st->minrun = oracle_minrun(n);
    for (uint64_t x = 0; x < n; ++x) perm[x] = (uint32_t)x;
    if (n == 0) { if (run_starts) run_starts[0] = 0; return 0; }

    uint32_t* bkey = (uint32_t*)malloc(n * sizeof(uint32_t));  /* stackBuf */
    uint32_t* bperm = (uint32_t*)malloc(n * sizeof(uint32_t));
    if (!bkey || !bperm) { free(bkey); free(bperm); return -1; }

    /* the run stack: (buffer = segment [si, sj) in stackBuf, power) */
    uint64_t stk_i[80], stk_j[80];
    uint32_t stk_p[80];
    int top = 0;

    uint64_t ci = 0, cj = extract_run(key, perm, 0, n, st->minrun, options, st); /* curr */
    if (run_starts) run_starts[0] = 0;
    st->runs = 1;
    while (cj < n) {                                   /* work not empty */
        uint64_t nj = cj, nk = extract_run(key, perm, cj, n, st->minrun, options, st); /* next */
        if (run_starts) run_starts[st->runs] = (uint32_t)nj;
        uint32_t p = oracle_power(n, ci, cj, nk);
        if (powers) powers[st->runs - 1] = (uint8_t)p;
        if (p > st->max_power) st->max_power = p;
        st->runs++;
        int in_stack = 0;
        while (top > 0 && stk_p[top - 1] >= p) {       /* merge top into curr */
            uint64_t ti = stk_i[top - 1];
            int last_pop = !(top > 1 && stk_p[top - 2] >= p);
            if (last_pop) {   /* result goes straight to stackBuf (Sec. 3) */
                pingpong_merge_to_stack(key, perm, bkey, bperm, ti, ci, cj, st);
                in_stack = 1;
            } else {
                pingpong_merge(key, perm, bkey, bperm, ti, ci, cj, st);
            }
            if (merges) {
                merges[3 * st->merges + 0] = (uint32_t)ti;
                merges[3 * st->merges + 1] = (uint32_t)ci;
                merges[3 * st->merges + 2] = (uint32_t)cj;
            }
            st->merges++;
            st->merge_cost += cj - ti;
            ci = ti;
            --top;                                     /* Pop */
        }
        /* Push (curr, p): an unmerged curr moves from input to stackBuf
         * (Sec. 3); this happens at most once per element. */
        if (!in_stack) {
            memcpy(bkey + ci, key + ci, (cj - ci) * sizeof(uint32_t));
            memcpy(bperm + ci, perm + ci, (cj - ci) * sizeof(uint32_t));
            st->moves += cj - ci;
        }
        stk_i[top] = ci; stk_j[top] = cj; stk_p[top] = p; ++top;
        if ((uint32_t)top > st->max_stack) st->max_stack = (uint32_t)top;
        ci = nj; cj = nk;                              /* curr <- next */
    }
    while (top > 0) {                                  /* final merges */
        uint64_t ti = stk_i[top - 1];
        pingpong_merge(key, perm, bkey, bperm, ti, ci, cj, st);
        if (merges) {
            merges[3 * st->merges + 0] = (uint32_t)ti;
            merges[3 * st->merges + 1] = (uint32_t)ci;
            merges[3 * st->merges + 2] = (uint32_t)cj;
        }
        st->merges++;
        st->merge_cost += cj - ti;
        ci = ti;
        --top;
    }
    (void)stk_j;
    if (run_starts) run_starts[st->runs] = (uint32_t)n;
    st->comparisons = st->scan_comparisons + st->merge_comparisons + st->insert_comparisons;
    free(bkey);
    free(bperm);
    return 0;
}

int oracle_powersort(uint32_t* key, uint32_t* perm, uint64_t n, uint32_t* run_starts,
                     uint8_t* powers, uint32_t* merges, oracle_stats* st)
{
    return oracle_powersort_ex(key, perm, n, run_starts, powers, merges, 0u, st);
}

/* ------------------------------------------------------------------------- */
/* Virtual-memory storage (Sec. 4).  Memory is managed in pages of P elements.
 * Physical page q < in_pages is input[qP, qP + P) (the last input page may be
 * partial and is never declared free); pages >= in_pages are extra pages,
 * allocated only when the free list is empty (Sec. 4 "Pages needed").  A
 * buffer is a deque over a list of pages; PopFront frees a page that becomes
 * empty, PushBack takes a page from the free list when its last page is full.
 * ExtractRun and MergeBuffers build a new buffer by PushBack while consuming
 * their inputs by PopFront (Sec. 4 operation list); the merge is Algorithm 2
 * done one element at a time, which frees and takes pages at exactly the
 * moments the page-by-page form (PageMerge) does. */
typedef struct {
    uint64_t P, n, in_pages, full_in_pages;
    uint64_t npages, cap_pages;        /* physical pages known so far */
    uint32_t** pkey;                   /* page storage (input pages alias input) */
    uint32_t** pperm;
    uint64_t* free_stack; uint64_t nfree;
    uint8_t* in_free;
    oracle_stats* st;
    int oom;
} vm_mem;

typedef struct {
    uint64_t* pages; uint64_t npages, cap;
    uint64_t head;   /* offset of the first element inside pages[0] */
    uint64_t len;
    int is_work;     /* the input buffer made by NewBuffer */
} vm_buf;

static void vm_buf_init(vm_buf* b) { memset(b, 0, sizeof(*b)); }
static void vm_buf_free(vm_buf* b) { free(b->pages); memset(b, 0, sizeof(*b)); }

static int vm_buf_append_page(vm_buf* b, uint64_t pg)
{
    if (b->npages == b->cap) {
        uint64_t nc = b->cap ? 2 * b->cap : 8;
        uint64_t* np = (uint64_t*)realloc(b->pages, nc * sizeof(uint64_t));
        if (!np) return -1;
        b->pages = np; b->cap = nc;
    }
    b->pages[b->npages++] = pg;
    return 0;
}

static uint64_t vm_take_page(vm_mem* m)
{
    if (m->nfree > 0) {
        uint64_t pg = m->free_stack[--m->nfree];
        m->in_free[pg] = 0;
        return pg;
    }
    if (m->npages == m->cap_pages) {                  /* grow the page table */
        uint64_t nc = 2 * m->cap_pages;
        uint32_t** nk = (uint32_t**)realloc(m->pkey, nc * sizeof(uint32_t*));
        if (!nk) { m->oom = 1; return 0; }
        m->pkey = nk;
        uint32_t** np = (uint32_t**)realloc(m->pperm, nc * sizeof(uint32_t*));
        if (!np) { m->oom = 1; return 0; }
        m->pperm = np;
        uint64_t* fs = (uint64_t*)realloc(m->free_stack, nc * sizeof(uint64_t));
        if (!fs) { m->oom = 1; return 0; }
        m->free_stack = fs;
        uint8_t* inf = (uint8_t*)realloc(m->in_free, nc);
        if (!inf) { m->oom = 1; return 0; }
        m->in_free = inf;
        m->cap_pages = nc;
    }
    uint64_t pg = m->npages++;
    m->pkey[pg] = (uint32_t*)malloc(m->P * sizeof(uint32_t));
    m->pperm[pg] = (uint32_t*)malloc(m->P * sizeof(uint32_t));
    if (!m->pkey[pg] || !m->pperm[pg]) m->oom = 1;
    m->in_free[pg] = 0;
    m->st->pool_pages++;
    return pg;
}

static void vm_give_page(vm_mem* m, uint64_t pg)
{
    m->free_stack[m->nfree++] = pg;
    m->in_free[pg] = 1;
}

static inline uint32_t* vm_kslot(vm_mem* m, const vm_buf* b, uint64_t x)
{
    uint64_t g = b->head + x;
    return &m->pkey[b->pages[g / m->P]][g % m->P];
}
static inline uint32_t* vm_pslot(vm_mem* m, const vm_buf* b, uint64_t x)
{
    uint64_t g = b->head + x;
    return &m->pperm[b->pages[g / m->P]][g % m->P];
}

/* PopFront: drop the first element; a full page that becomes empty goes to
 * the free list.  The partial last input page is never freed. */
static void vm_pop_front(vm_mem* m, vm_buf* b)
{
    b->head++; b->len--;
    if (b->head == m->P) {
        uint64_t pg = b->pages[0];
        memmove(b->pages, b->pages + 1, (b->npages - 1) * sizeof(uint64_t));
        b->npages--;
        b->head = 0;
        if (!(pg >= m->full_in_pages && pg < m->in_pages)) vm_give_page(m, pg);
    } else if (b->len == 0 && b->is_work) {
        /* the work buffer ends inside the partial input page: keep it */
    }
}

static int vm_push_back(vm_mem* m, vm_buf* b, uint32_t k, uint32_t p)
{
    if (b->head + b->len == b->npages * m->P) {
        uint64_t pg = vm_take_page(m);
        if (m->oom || vm_buf_append_page(b, pg)) return -1;
    }
    *vm_kslot(m, b, b->len) = k;
    *vm_pslot(m, b, b->len) = p;
    b->len++;
    m->st->moves++;
    return 0;
}

static uint64_t vm_pages_in_use(const vm_mem* m) { return m->npages - m->nfree; }

static void vm_note_peak(vm_mem* m)
{
    uint64_t u = vm_pages_in_use(m);
    if (u > m->st->peak_pages) m->st->peak_pages = u;
}

/* ExtractRun on the VM work buffer: find the run in place (as in the
 * Pingpong form; with ORACLE_DESCENDING_RUNS a strictly decreasing run is
 * reversed in place), sort a forced run by insertion sort in place, then move
 * it element by element into a fresh buffer. */
static int vm_extract_run(vm_mem* m, vm_buf* work, vm_buf* out, uint32_t minrun, uint32_t options)
{
    oracle_stats* st = m->st;
    uint64_t avail = work->len, e = 1;
    int down = 0;
    if ((options & ORACLE_DESCENDING_RUNS) && e < avail) {
        st->scan_comparisons++;
        down = key_gt(*vm_kslot(m, work, 0), *vm_kslot(m, work, 1));
        ++e;
    }
    while (e < avail) {
        st->scan_comparisons++;
        const int desc = key_gt(*vm_kslot(m, work, e - 1), *vm_kslot(m, work, e));
        if (desc != down) break;   /* ascending: first descent; decreasing: first non-descent */
        ++e;
    }
    if (down) {
        for (uint64_t x = 0, y = e - 1; x < y; ++x, --y) {
            uint32_t tk = *vm_kslot(m, work, x), tp = *vm_pslot(m, work, x);
            *vm_kslot(m, work, x) = *vm_kslot(m, work, y);
            *vm_pslot(m, work, x) = *vm_pslot(m, work, y);
            *vm_kslot(m, work, y) = tk;
            *vm_pslot(m, work, y) = tp;
            st->reverse_moves += 2;
        }
        st->reversed_runs++;
    }
    if (e < minrun) {
        uint64_t end = minrun < avail ? minrun : avail;
        for (uint64_t x = e; x < end; ++x) {
            uint32_t v = *vm_kslot(m, work, x), pv = *vm_pslot(m, work, x);
            uint64_t y = x;
            while (y > 0) {
                st->insert_comparisons++;
                if (!key_gt(*vm_kslot(m, work, y - 1), v)) break;
                *vm_kslot(m, work, y) = *vm_kslot(m, work, y - 1);
                *vm_pslot(m, work, y) = *vm_pslot(m, work, y - 1);
                st->insert_moves++;
                --y;
            }
            if (y != x) { *vm_kslot(m, work, y) = v; *vm_pslot(m, work, y) = pv; st->insert_moves++; }
        }
        e = end;
    }
    vm_buf_init(out);
    for (uint64_t x = 0; x < e; ++x) {
        uint32_t k = *vm_kslot(m, work, 0), p = *vm_pslot(m, work, 0);
        vm_pop_front(m, work);
        if (vm_push_back(m, out, k, p)) return -1;
        vm_note_peak(m);
    }
    return 0;
}

/* MergeBuffers(a, b): Algorithm 2 with PopFront / PushBack; ties take a. */
static int vm_merge(vm_mem* m, vm_buf* a, vm_buf* b, vm_buf* out)
{
    vm_buf_init(out);
    while (a->len && b->len) {
        m->st->merge_comparisons++;
        vm_buf* src = !key_gt(*vm_kslot(m, a, 0), *vm_kslot(m, b, 0)) ? a : b;
        uint32_t k = *vm_kslot(m, src, 0), p = *vm_pslot(m, src, 0);
        vm_pop_front(m, src);
        if (vm_push_back(m, out, k, p)) return -1;
        vm_note_peak(m);
    }
    vm_buf* rest = a->len ? a : b;
    while (rest->len) {
        uint32_t k = *vm_kslot(m, rest, 0), p = *vm_pslot(m, rest, 0);
        vm_pop_front(m, rest);
        if (vm_push_back(m, out, k, p)) return -1;
        vm_note_peak(m);
    }
    /* a and b are empty; their last (partial) pages are released */
    for (int s = 0; s < 2; ++s) {
        vm_buf* z = s ? b : a;
        for (uint64_t q = 0; q < z->npages; ++q) {
            uint64_t pg = z->pages[q];
            if (!(pg >= m->full_in_pages && pg < m->in_pages)) vm_give_page(m, pg);
        }
        vm_buf_free(z);
    }
    return 0;
}

/* Copy(curr, input) (Sec. 4): walk the logical pages of curr in order; if the
 * input page that must receive logical page q is still used by a later
 * logical page, that page is first moved out to a free page; then logical
 * page q is copied into place.  The search is linear, as in the paper. */
static int vm_copy_back(vm_mem* m, vm_buf* c)
{
    uint64_t P = m->P;
    for (uint64_t q = 0; q < c->npages; ++q) {
        uint64_t src = c->pages[q];
        if (src == q) continue;
        if (m->in_free[q]) {                     /* target is free: claim it */
            for (uint64_t f = 0; f < m->nfree; ++f)
                if (m->free_stack[f] == q) { m->free_stack[f] = m->free_stack[--m->nfree]; break; }
            m->in_free[q] = 0;
        }
        for (uint64_t r = q + 1; r < c->npages; ++r) {
            if (c->pages[r] == q) {              /* evict page q first */
                uint64_t pg = vm_take_page(m);
                if (m->oom) return -1;
                uint64_t cnt = (r + 1 == c->npages) ? c->len - r * P : P;
                memcpy(m->pkey[pg], m->pkey[q], cnt * sizeof(uint32_t));
                memcpy(m->pperm[pg], m->pperm[q], cnt * sizeof(uint32_t));
                m->st->moves += cnt;
                c->pages[r] = pg;
                vm_note_peak(m);
                break;
            }
        }
        uint64_t cnt = (q + 1 == c->npages) ? c->len - q * P : P;
        memcpy(m->pkey[q], m->pkey[src], cnt * sizeof(uint32_t));
        memcpy(m->pperm[q], m->pperm[src], cnt * sizeof(uint32_t));
        m->st->moves += cnt;
        c->pages[q] = q;
        vm_give_page(m, src);
    }
    return 0;
}

/* Algorithm 1 with virtual-memory buffers.  Same outputs as oracle_powersort
 * plus st->peak_pages (pages in use at the busiest moment, input pages
 * included) and st->pool_pages (pages allocated beyond the input).
 * page_size must be >= 1; options as for oracle_powersort_ex.  Returns 0,
 * or -1 on allocation failure. */
int oracle_powersort_vm_ex(uint32_t* key, uint32_t* perm, uint64_t n, uint64_t page_size,
                           uint32_t* run_starts, uint8_t* powers, uint32_t* merges,
                           uint32_t options, oracle_stats* st)
{
    memset(st, 0, sizeof(*st));
    g_key_order = options & (ORACLE_KEY_I32 | ORACLE_KEY_F32 | ORACLE_RECORDS | ORACLE_KEYS64);
    st->n = n;
    st->minrun = oracle_minrun(n);
    st->page_size = (uint32_t)page_size;
    for (uint64_t x = 0; x < n; ++x) perm[x] = (uint32_t)x;
    if (n == 0) { if (run_starts) run_starts[0] = 0; return 0; }
    if (page_size == 0) return -1;

    vm_mem m;
    memset(&m, 0, sizeof(m));
    m.P = page_size; m.n = n; m.st = st;
    m.full_in_pages = n / page_size;
    m.in_pages = (n + page_size - 1) / page_size;
    m.cap_pages = m.in_pages + 64;
    m.npages = m.in_pages;
    m.pkey = (uint32_t**)malloc(m.cap_pages * sizeof(uint32_t*));
    m.pperm = (uint32_t**)malloc(m.cap_pages * sizeof(uint32_t*));
    m.free_stack = (uint64_t*)malloc(m.cap_pages * sizeof(uint64_t));
    m.in_free = (uint8_t*)calloc(m.cap_pages, 1);
    int rc = -1;
    vm_buf work, curr, next, stk[80];
    uint32_t stk_p[80];
    int top = 0;
    vm_buf_init(&work); vm_buf_init(&curr); vm_buf_init(&next);
    if (!m.pkey || !m.pperm || !m.free_stack || !m.in_free) goto done;
    for (uint64_t q = 0; q < m.in_pages; ++q) { m.pkey[q] = key + q * page_size; m.pperm[q] = perm + q * page_size; }

    /* NewBuffer(input): segment the input into pages */
    work.is_work = 1;
    for (uint64_t q = 0; q < m.in_pages; ++q) if (vm_buf_append_page(&work, q)) goto done;
    work.len = n;
    vm_note_peak(&m);

    uint64_t ci = 0;
    if (vm_extract_run(&m, &work, &curr, st->minrun, options)) goto done;
    uint64_t cj = curr.len;
    if (run_starts) run_starts[0] = 0;
    st->runs = 1;
    while (work.len) {
        uint64_t nj = cj;
        if (vm_extract_run(&m, &work, &next, st->minrun, options)) goto done;
        uint64_t nk = nj + next.len;
        if (run_starts) run_starts[st->runs] = (uint32_t)nj;
        uint32_t p = oracle_power(n, ci, cj, nk);
        if (powers) powers[st->runs - 1] = (uint8_t)p;
        if (p > st->max_power) st->max_power = p;
        st->runs++;
        while (top > 0 && stk_p[top - 1] >= p) {
            uint64_t ti = cj - curr.len - stk[top - 1].len;
            vm_buf res;
            if (vm_merge(&m, &stk[top - 1], &curr, &res)) goto done;
            if (merges) {
                merges[3 * st->merges + 0] = (uint32_t)ti;
                merges[3 * st->merges + 1] = (uint32_t)ci;
                merges[3 * st->merges + 2] = (uint32_t)cj;
            }
            st->merges++;
            st->merge_cost += cj - ti;
            curr = res;
            ci = ti;
            --top;
        }
        stk[top] = curr; stk_p[top] = p; ++top;          /* Push: metadata only */
        if ((uint32_t)top > st->max_stack) st->max_stack = (uint32_t)top;
        curr = next; vm_buf_init(&next);
        ci = nj; cj = nk;
    }
    while (top > 0) {
        uint64_t ti = cj - curr.len - stk[top - 1].len;
        vm_buf res;
        if (vm_merge(&m, &stk[top - 1], &curr, &res)) goto done;
        if (merges) {
            merges[3 * st->merges + 0] = (uint32_t)ti;
            merges[3 * st->merges + 1] = (uint32_t)ci;
            merges[3 * st->merges + 2] = (uint32_t)cj;
        }
        st->merges++;
        st->merge_cost += cj - ti;
        curr = res;
        ci = ti;
        --top;
    }
    if (run_starts) run_starts[st->runs] = (uint32_t)n;
    if (vm_copy_back(&m, &curr)) goto done;            /* Copy(curr, input) */
    st->comparisons = st->scan_comparisons + st->merge_comparisons + st->insert_comparisons;
    rc = m.oom ? -1 : 0;
done:
    vm_buf_free(&work); vm_buf_free(&curr); vm_buf_free(&next);
    for (int s = 0; s < top; ++s) vm_buf_free(&stk[s]);
    if (m.pkey) for (uint64_t q = m.in_pages; q < m.npages; ++q) { free(m.pkey[q]); free(m.pperm[q]); }
    free(m.pkey); free(m.pperm); free(m.free_stack); free(m.in_free);
    return rc;
}

int oracle_powersort_vm(uint32_t* key, uint32_t* perm, uint64_t n, uint64_t page_size,
                        uint32_t* run_starts, uint8_t* powers, uint32_t* merges,
                        oracle_stats* st)
{
    return oracle_powersort_vm_ex(key, perm, n, page_size, run_starts, powers, merges, 0u, st);
}

/* Records (ORACLE_RECORDS): Algorithm 1 on the record indices 0..n-1, every
 * comparison made on the rows.  perm receives the stable order (perm[r] =
 * index of the r-th record); run_starts, powers, merges and st as for
 * oracle_powersort_ex (options may add ORACLE_DESCENDING_RUNS). */
int oracle_powersort_records(const uint32_t* rec, uint32_t words, uint64_t n, uint32_t* perm,
                             uint32_t* run_starts, uint8_t* powers, uint32_t* merges, uint32_t options,
                             oracle_stats* st)
{
    uint32_t* idx = (uint32_t*)malloc((n ? n : 1) * sizeof(uint32_t));
    if (!idx) return -1;
    for (uint64_t i = 0; i < n; ++i) idx[i] = (uint32_t)i;
    g_rec = rec;
    g_rec_words = words;
    int rc = oracle_powersort_ex(idx, perm, n, run_starts, powers, merges, options | ORACLE_RECORDS, st);
    free(idx);
    return rc;
}

/* The definition for records: indices ordered by (row, index). */
int oracle_stable_sort_records(const uint32_t* rec, uint32_t words, uint64_t n, uint32_t* perm_out)
{
    uint32_t* idx = (uint32_t*)malloc((n ? n : 1) * sizeof(uint32_t));
    if (!idx) return -1;
    for (uint64_t i = 0; i < n; ++i) idx[i] = (uint32_t)i;
    g_rec = rec;
    g_rec_words = words;
    int rc = oracle_stable_sort_ex(idx, n, ORACLE_RECORDS, NULL, perm_out);
    free(idx);
    return rc;
}

/* 64-bit keys: Algorithm 1 on the indices 0..n-1, comparing keys[i] by the
 * order `options` names (0: unsigned, ORACLE_KEY_I32: int64, ORACLE_KEY_F32:
 * binary64 totalOrder; ORACLE_DESCENDING_RUNS may be added).  perm receives
 * the stable order. */
int oracle_powersort_keys64(const uint64_t* keys, uint64_t n, uint32_t* perm, uint32_t* run_starts,
                            uint8_t* powers, uint32_t* merges, uint32_t options, oracle_stats* st)
{
    uint32_t* idx = (uint32_t*)malloc((n ? n : 1) * sizeof(uint32_t));
    if (!idx) return -1;
    for (uint64_t i = 0; i < n; ++i) idx[i] = (uint32_t)i;
    g_keys64 = keys;
    int rc = oracle_powersort_ex(idx, perm, n, run_starts, powers, merges, options | ORACLE_KEYS64, st);
    free(idx);
    return rc;
}
