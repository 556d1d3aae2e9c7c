/*
 * FP64 oracle of the CHERT traveltime relaxation -- TEST INFRASTRUCTURE ONLY.
 * Only tests, the smoke check and the benchmark's CPU-baseline leg load this.
 *
 * Graph (the nodal ray network of the paper's "Grid and Nodal Ray-Network
 * Representation"): nodes on an nx*ny*nz lattice, node = x + nx*(y + ny*z),
 * spacing dx; a directed edge i -> j = i + o for every stencil offset o that
 * stays inside the lattice.
 *
 * Edge increments (Eq. 27-30): with L = dx*|o| and sel[k][o] the value that
 * the direction lookup picked for class k and offset o,
 *   propagation (component 0): w = L / (0.5*(V[k_i][o] + V[k_j][o]))
 *   attenuation (component 1): w = L * (0.5*(A[k_i][o] + A[k_j][o]))
 * The two components are separate shortest-path problems (Eq. 31).
 *
 * The fixed point of Eq. 31 from tau(src) = 0 is computed with textbook
 * Dijkstra on a binary heap (lazy deletion).  Parents follow the
 * deterministic rule par_j = argmin_i (tau_i + w_ij), ties to the smallest i;
 * the source is its own parent and an unreachable node has par = -1 and
 * tau = +inf (Eq. 33).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

typedef struct {
    double key;
    int64_t node;
} heap_item;

typedef struct {
    heap_item* a;
    int64_t n, cap;
} heap;

static int heap_push(heap* h, double key, int64_t node) {
    if (h->n == h->cap) {
        int64_t cap = h->cap ? 2 * h->cap : 1024;
        heap_item* a = (heap_item*)realloc(h->a, (size_t)cap * sizeof(heap_item));
        if (!a) return -1;
        h->a = a;
        h->cap = cap;
    }
    int64_t i = h->n++;
    while (i > 0) {
        int64_t parent = (i - 1) / 2;
        if (h->a[parent].key <= key) break;
        h->a[i] = h->a[parent];
        i = parent;
    }
    h->a[i].key = key;
    h->a[i].node = node;
    return 0;
}

static heap_item heap_pop(heap* h) {
    heap_item top = h->a[0];
    heap_item last = h->a[--h->n];
    int64_t i = 0;
    for (;;) {
        int64_t c = 2 * i + 1;
        if (c >= h->n) break;
        if (c + 1 < h->n && h->a[c + 1].key < h->a[c].key) c++;
        if (last.key <= h->a[c].key) break;
        h->a[i] = h->a[c];
        i = c;
    }
    if (h->n > 0) h->a[i] = last;
    return top;
}

static double edge_weight(int component, double L, const double* sel, int n_off,
                          int32_t ki, int32_t kj, int o) {
    double a = sel[(size_t)ki * n_off + o];
    double b = sel[(size_t)kj * n_off + o];
    if (component == 0) return L / (0.5 * (a + b));
    return L * (0.5 * (a + b));
}

/* Neighbour of node (x,y,z) through offset o, or -1 outside the lattice. */
static int64_t step(int64_t nx, int64_t ny, int64_t nz, int64_t x, int64_t y, int64_t z,
                    const int32_t* off, int o, int sign) {
    int64_t X = x + sign * off[3 * o], Y = y + sign * off[3 * o + 1], Z = z + sign * off[3 * o + 2];
    if (X < 0 || X >= nx || Y < 0 || Y >= ny || Z < 0 || Z >= nz) return -1;
    return X + nx * (Y + ny * Z);
}

/* Returns 0, or -1 on a bad argument / allocation failure. */
int oracle_dijkstra(int64_t nx, int64_t ny, int64_t nz, double dx,
                    const int32_t* cls, const int32_t* off, int n_off,
                    const double* sel, int component, int64_t src,
                    double* tau, int32_t* par) {
    int64_t n = nx * ny * nz;
    if (n <= 0 || src < 0 || src >= n || n_off <= 0) return -1;
    double* L = (double*)malloc((size_t)n_off * sizeof(double));
    char* done = (char*)calloc((size_t)n, 1);
    heap h = {0, 0, 0};
    if (!L || !done) { free(L); free(done); return -1; }
    for (int o = 0; o < n_off; o++) {
        double ox = off[3 * o], oy = off[3 * o + 1], oz = off[3 * o + 2];
        L[o] = dx * sqrt(ox * ox + oy * oy + oz * oz);
    }
    for (int64_t i = 0; i < n; i++) { tau[i] = INFINITY; par[i] = -1; }
    tau[src] = 0.0;
    if (heap_push(&h, 0.0, src)) goto fail;
    while (h.n > 0) {
        heap_item it = heap_pop(&h);
        int64_t u = it.node;
        if (done[u] || it.key > tau[u]) continue;
        done[u] = 1;
        int64_t ux = u % nx, uy = (u / nx) % ny, uz = u / (nx * ny);
        for (int o = 0; o < n_off; o++) {
            int64_t v = step(nx, ny, nz, ux, uy, uz, off, o, +1);
            if (v < 0 || done[v]) continue;
            double w = edge_weight(component, L[o], sel, n_off, cls[u], cls[v], o);
            if (!(w >= 0.0) || isinf(w)) continue;      /* no cache entry: no edge */
            double t = tau[u] + w;
            if (t < tau[v]) {
                tau[v] = t;
                if (heap_push(&h, t, v)) goto fail;
            }
        }
    }
    /* parents: argmin over in-neighbours, ties to the smallest node index */
    for (int64_t j = 0; j < n; j++) {
        if (j == src) { par[j] = (int32_t)src; continue; }
        if (isinf(tau[j])) { par[j] = -1; continue; }
        int64_t jx = j % nx, jy = (j / nx) % ny, jz = j / (nx * ny);
        double best = INFINITY;
        int64_t bi = -1;
        for (int o = 0; o < n_off; o++) {
            int64_t i = step(nx, ny, nz, jx, jy, jz, off, o, -1);
            if (i < 0 || isinf(tau[i])) continue;
            double w = edge_weight(component, L[o], sel, n_off, cls[i], cls[j], o);
            if (!(w >= 0.0) || isinf(w)) continue;
            double c = tau[i] + w;
            if (c < best || (c == best && i < bi)) { best = c; bi = i; }
        }
        par[j] = (int32_t)bi;
    }
    free(h.a); free(L); free(done);
    return 0;
fail:
    free(h.a); free(L); free(done);
    return -1;
}
