/*
 * oracle.c -- FP64 CPU oracle for sliced bucket elimination.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library. It shares no code,
 * header, table or helper with the CUDA path; the two meet only through the
 * seeded gate lists of the input generator and through plain integer arrays
 * (an elimination order and a sliced set, given as (qubit, segment) keys).
 *
 * What it computes, in plain double-precision complex arithmetic:
 *  - orc_statevector: the textbook state vector C|0^n> (basis index
 *    sum_q x_q 2^q), applying each gate to pairs of amplitudes. Independent of
 *    the network construction; used as the brute-force pin.
 *  - orc_network_*: the circuit's graphical-model network (Section II.A:
 *    variables are vertices, each tensor is a clique, single-variable tensors
 *    are self-loops). Reading of the circuit construction, which the paper
 *    only cites: every non-diagonal one-qubit gate U adds a tensor
 *    U[v_new, v_old] and starts a new variable on its wire; a diagonal gate
 *    adds a tensor on the wire's current variable; CZ adds (-1)^(a b) on the
 *    two current variables; the input variables are fixed to 0 and the output
 *    variables to the bitstring.
 *  - orc_contract_slice: bucket elimination, Eq. 2: for every variable u of
 *    the order, multiply all tensors that contain u, sum over u, and put the
 *    result back (a rank-0 result multiplies the running scalar). Slicing
 *    (Eq. 4) fixes each variable of mu to the bit of the slice index.
 *  - orc_contract_sum: Eq. 5, the sum of the slice results in increasing s.
 *
 * Every bucket's multiplications and additions are counted (complex ops), so
 * a test can compare a cost model against the operations actually done.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cx;

enum { K_H = 0, K_X12 = 1, K_Y12 = 2, K_T = 3, K_CZ = 4, K_CNOT = 5, K_U1 = 6 };

/* ---- gate matrices: U[row = output value][column = input value] ------- */
static int gate_matrix(int kind, const double* m, cx U[2][2]) {
  const double s = 1.0 / sqrt(2.0);
  switch (kind) {
    case K_H:
      U[0][0] = s; U[0][1] = s; U[1][0] = s; U[1][1] = -s;
      return 1;
    case K_X12: /* R_x(pi/2) = (1/sqrt2)[[1, -i], [-i, 1]] */
      U[0][0] = s; U[0][1] = -I * s; U[1][0] = -I * s; U[1][1] = s;
      return 1;
    case K_Y12: /* R_y(pi/2) = (1/sqrt2)[[1, -1], [1, 1]] */
      U[0][0] = s; U[0][1] = -s; U[1][0] = s; U[1][1] = s;
      return 1;
    case K_T:
      U[0][0] = 1; U[0][1] = 0; U[1][0] = 0; U[1][1] = cexp(I * M_PI / 4.0);
      return 1;
    case K_U1:
      U[0][0] = m[0] + I * m[1]; U[0][1] = m[2] + I * m[3];
      U[1][0] = m[4] + I * m[5]; U[1][1] = m[6] + I * m[7];
      return 1;
    default:
      return 0;
  }
}

static int is_diag_1q(int kind) { return kind == K_T; }

/* ---- brute-force state vector ------------------------------------------ */
static void sv_apply_1q(cx* psi, int n, int q, cx U[2][2]) {
  const uint64_t dim = 1ull << n, bit = 1ull << q;
  for (uint64_t i = 0; i < dim; ++i) {
    if (i & bit) continue;
    cx a0 = psi[i], a1 = psi[i | bit];
    psi[i] = U[0][0] * a0 + U[0][1] * a1;
    psi[i | bit] = U[1][0] * a0 + U[1][1] * a1;
  }
}

/* psi (2^n complex as re,im pairs) = C |0^n>. Returns 0 on success. */
int orc_statevector(int n, size_t n_gates, const int* kind, const int* q0, const int* q1,
                    const double* mats, double* psi_out) {
  if (n < 1 || n > 30) return 1;
  const uint64_t dim = 1ull << n;
  cx* psi = (cx*)calloc(dim, sizeof(cx));
  if (!psi) return 2;
  psi[0] = 1.0;
  for (size_t g = 0; g < n_gates; ++g) {
    const int k = kind[g];
    if (k == K_CZ) {
      const uint64_t a = 1ull << q0[g], b = 1ull << q1[g];
      for (uint64_t i = 0; i < dim; ++i)
        if ((i & a) && (i & b)) psi[i] = -psi[i];
    } else if (k == K_CNOT) { /* swap the target bit where the control is 1 */
      const uint64_t c = 1ull << q0[g], t = 1ull << q1[g];
      for (uint64_t i = 0; i < dim; ++i)
        if ((i & c) && !(i & t)) {
          cx tmp = psi[i];
          psi[i] = psi[i | t];
          psi[i | t] = tmp;
        }
    } else {
      cx U[2][2];
      if (!gate_matrix(k, mats + 8 * g, U)) { free(psi); return 3; }
      sv_apply_1q(psi, n, q0[g], U);
    }
  }
  for (uint64_t i = 0; i < dim; ++i) {
    psi_out[2 * i] = creal(psi[i]);
    psi_out[2 * i + 1] = cimag(psi[i]);
  }
  free(psi);
  return 0;
}

/* ---- network ------------------------------------------------------------ */
typedef struct {
  int rank;       /* number of variables */
  int* vars;      /* oracle variable ids */
  cx* val;        /* 2^rank entries; entry of assignment a is sum_i a_i 2^i */
} otensor;

typedef struct {
  int n_qubits;
  int n_vars;
  int* var_qubit;
  int* var_seg;
  int* is_input;   /* segment 0 */
  int* is_output;  /* last segment of its qubit */
  int n_tensors;
  otensor* t;
  int cap_t;
} onet;

static int add_var(onet* N, int q, int seg) {
  int id = N->n_vars++;
  N->var_qubit = (int*)realloc(N->var_qubit, sizeof(int) * N->n_vars);
  N->var_seg = (int*)realloc(N->var_seg, sizeof(int) * N->n_vars);
  N->is_input = (int*)realloc(N->is_input, sizeof(int) * N->n_vars);
  N->is_output = (int*)realloc(N->is_output, sizeof(int) * N->n_vars);
  N->var_qubit[id] = q;
  N->var_seg[id] = seg;
  N->is_input[id] = (seg == 0);
  N->is_output[id] = 0;
  return id;
}

static otensor* add_tensor(onet* N, int rank) {
  if (N->n_tensors == N->cap_t) {
    N->cap_t = N->cap_t ? 2 * N->cap_t : 64;
    N->t = (otensor*)realloc(N->t, sizeof(otensor) * N->cap_t);
  }
  otensor* T = &N->t[N->n_tensors++];
  T->rank = rank;
  T->vars = (int*)malloc(sizeof(int) * (rank ? rank : 1));
  T->val = (cx*)calloc((size_t)1 << rank, sizeof(cx));
  return T;
}

static void free_net(onet* N) {
  for (int i = 0; i < N->n_tensors; ++i) { free(N->t[i].vars); free(N->t[i].val); }
  free(N->t); free(N->var_qubit); free(N->var_seg); free(N->is_input); free(N->is_output);
  free(N);
}

/* Adds a non-diagonal one-qubit gate U on qubit q: tensor U[v_new, v_old]. */
static void net_nondiag(onet* N, int* cur, int* seg, int q, cx U[2][2]) {
  int vold = cur[q];
  int vnew = add_var(N, q, ++seg[q]);
  otensor* T = add_tensor(N, 2);
  T->vars[0] = vnew; T->vars[1] = vold;
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) T->val[a + 2 * b] = U[a][b];
  cur[q] = vnew;
}

static void net_cz(onet* N, const int* cur, int qa, int qb) {
  otensor* T = add_tensor(N, 2);
  T->vars[0] = cur[qa]; T->vars[1] = cur[qb];
  T->val[0] = 1; T->val[1] = 1; T->val[2] = 1; T->val[3] = -1;
}

static onet* build_net(int n, size_t n_gates, const int* kind, const int* q0, const int* q1,
                       const double* mats) {
  onet* N = (onet*)calloc(1, sizeof(onet));
  N->n_qubits = n;
  int* cur = (int*)malloc(sizeof(int) * n);
  int* seg = (int*)calloc(n, sizeof(int));
  for (int q = 0; q < n; ++q) cur[q] = add_var(N, q, 0);
  for (size_t g = 0; g < n_gates; ++g) {
    const int k = kind[g];
    if (k == K_CZ) {
      net_cz(N, cur, q0[g], q1[g]);
    } else if (k == K_CNOT) { /* H(t) CZ(c,t) H(t) */
      cx Hm[2][2];
      gate_matrix(K_H, NULL, Hm);
      net_nondiag(N, cur, seg, q1[g], Hm);
      net_cz(N, cur, q0[g], q1[g]);
      net_nondiag(N, cur, seg, q1[g], Hm);
    } else {
      cx U[2][2];
      if (!gate_matrix(k, mats + 8 * g, U)) { free(cur); free(seg); free_net(N); return NULL; }
      if (is_diag_1q(k)) {
        otensor* T = add_tensor(N, 1);
        T->vars[0] = cur[q0[g]];
        T->val[0] = U[0][0]; T->val[1] = U[1][1];
      } else {
        net_nondiag(N, cur, seg, q0[g], U);
      }
    }
  }
  for (int q = 0; q < n; ++q) N->is_output[cur[q]] = 1;
  free(cur); free(seg);
  return N;
}

/* Number of free variables and their keys (qubit, segment), in creation order. */
int orc_network_vars(int n, size_t n_gates, const int* kind, const int* q0, const int* q1,
                     const double* mats, int* out_qubit, int* out_seg, int cap) {
  onet* N = build_net(n, n_gates, kind, q0, q1, mats);
  if (!N) return -1;
  int c = 0;
  for (int v = 0; v < N->n_vars; ++v) {
    if (N->is_input[v] || N->is_output[v]) continue;
    if (c < cap) { out_qubit[c] = N->var_qubit[v]; out_seg[c] = N->var_seg[v]; }
    ++c;
  }
  free_net(N);
  return c;
}

/* Edges of the free-variable graph (pairs of indices into the orc_network_vars
 * list) and the number of leaf tensors after fixing. Returns #edges or -1. */
int orc_network_graph(int n, size_t n_gates, const int* kind, const int* q0, const int* q1,
                      const double* mats, int* out_edges, int cap_edges) {
  onet* N = build_net(n, n_gates, kind, q0, q1, mats);
  if (!N) return -1;
  int* fid = (int*)malloc(sizeof(int) * N->n_vars);
  int nf = 0;
  for (int v = 0; v < N->n_vars; ++v) fid[v] = (N->is_input[v] || N->is_output[v]) ? -1 : nf++;
  int ne = 0;
  for (int i = 0; i < N->n_tensors; ++i) {
    otensor* T = &N->t[i];
    for (int a = 0; a < T->rank; ++a)
      for (int b = a + 1; b < T->rank; ++b) {
        int x = fid[T->vars[a]], y = fid[T->vars[b]];
        if (x < 0 || y < 0 || x == y) continue;
        if (ne < cap_edges) { out_edges[2 * ne] = x; out_edges[2 * ne + 1] = y; }
        ++ne;
      }
  }
  free(fid);
  free_net(N);
  return ne;
}

/* ---- bucket elimination ------------------------------------------------- */
typedef struct {
  double cmul;  /* complex multiplications */
  double cadd;  /* complex additions */
} ocount;

/* Restricts tensor T by the fixed values fixed[v] (-1 = free). */
static otensor restrict_tensor(const otensor* T, const int* fixed) {
  otensor R;
  int nf = 0;
  for (int i = 0; i < T->rank; ++i) nf += (fixed[T->vars[i]] < 0);
  R.rank = nf;
  R.vars = (int*)malloc(sizeof(int) * (nf ? nf : 1));
  R.val = (cx*)calloc((size_t)1 << nf, sizeof(cx));
  int c = 0;
  for (int i = 0; i < T->rank; ++i)
    if (fixed[T->vars[i]] < 0) R.vars[c++] = T->vars[i];
  for (uint64_t a = 0; a < (1ull << nf); ++a) {
    /* full assignment of T: free positions from a, fixed ones from `fixed` */
    uint64_t full = 0;
    int fpos = 0;
    for (int i = 0; i < T->rank; ++i) {
      int v = T->vars[i];
      int bit = fixed[v] >= 0 ? fixed[v] : (int)((a >> fpos++) & 1);
      full |= (uint64_t)bit << i;
    }
    R.val[a] = T->val[full];
  }
  return R;
}

static int contains(const otensor* T, int v) {
  for (int i = 0; i < T->rank; ++i)
    if (T->vars[i] == v) return 1;
  return 0;
}

/*
 * One slice: fixes input wires to 0, output wires to bits[q], mu_j to bit j
 * of s, then eliminates the free variables in `order` (oracle variable ids).
 * Returns 0 and the slice value in *out, or nonzero on a malformed order.
 */
static int contract_slice(const onet* N, const uint8_t* bits, const int* order, int n_order,
                          const int* mu, int p, uint64_t s, cx* out, ocount* cnt) {
  int* fixed = (int*)malloc(sizeof(int) * N->n_vars);
  cx acc = 1.0;
  for (int v = 0; v < N->n_vars; ++v) {
    fixed[v] = -1;
    if (N->is_input[v]) fixed[v] = 0;
    if (N->is_output[v]) {
      int x = bits[N->var_qubit[v]] ? 1 : 0;
      if (N->is_input[v] && x != 0) acc = 0.0; /* wire with no non-diagonal gate: <x|0> */
      if (!N->is_input[v]) fixed[v] = x;
    }
  }
  for (int j = 0; j < p; ++j) fixed[mu[j]] = (int)((s >> j) & 1);

  /* every free variable appears in the order exactly once */
  int* seen = (int*)calloc(N->n_vars, sizeof(int));
  for (int i = 0; i < n_order; ++i) {
    int v = order[i];
    if (v < 0 || v >= N->n_vars || fixed[v] >= 0 || seen[v]) { free(seen); free(fixed); return 1; }
    seen[v] = 1;
  }
  for (int v = 0; v < N->n_vars; ++v)
    if (fixed[v] < 0 && !seen[v]) { free(seen); free(fixed); return 1; }
  free(seen);

  int cap = N->n_tensors + n_order + 1, np = 0;
  otensor* pool = (otensor*)malloc(sizeof(otensor) * cap);
  for (int i = 0; i < N->n_tensors; ++i) {
    otensor R = restrict_tensor(&N->t[i], fixed);
    if (R.rank == 0) { acc *= R.val[0]; free(R.vars); free(R.val); }
    else pool[np++] = R;
  }

  for (int step = 0; step < n_order; ++step) {
    const int u = order[step];
    /* the bucket of u: every remaining tensor that contains u */
    int* sel = (int*)malloc(sizeof(int) * (np ? np : 1));
    int ns = 0;
    for (int i = 0; i < np; ++i)
      if (contains(&pool[i], u)) sel[ns++] = i;
    if (ns == 0) { /* u appears in no tensor: summing it doubles the result */
      acc *= 2.0;
      free(sel);
      continue;
    }
    /* union of the bucket's variables, u first */
    int* uni = (int*)malloc(sizeof(int) * 64);
    int nu = 0;
    uni[nu++] = u;
    for (int a = 0; a < ns; ++a) {
      otensor* T = &pool[sel[a]];
      for (int i = 0; i < T->rank; ++i) {
        int v = T->vars[i], dup = 0;
        for (int b = 0; b < nu; ++b) dup |= (uni[b] == v);
        if (!dup) {
          if (nu == 64) { free(uni); free(sel); free(fixed); return 2; }
          uni[nu++] = v;
        }
      }
    }
    /* position of each tensor variable inside the union */
    int** pos = (int**)malloc(sizeof(int*) * (size_t)(ns > 0 ? ns : 1));
    for (int a = 0; a < ns; ++a) {
      otensor* T = &pool[sel[a]];
      pos[a] = (int*)malloc(sizeof(int) * T->rank);
      for (int i = 0; i < T->rank; ++i)
        for (int b = 0; b < nu; ++b)
          if (uni[b] == T->vars[i]) pos[a][i] = b;
    }
    /* result over uni[1..nu-1]: out[b] = sum_{u in {0,1}} prod_j T_j[(u, b) restricted] */
    const int ro = nu - 1;
    const uint64_t nout = 1ull << ro;
    cx* res = (cx*)malloc(sizeof(cx) * nout);
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < (int64_t)nout; ++b) {
      cx term[2];
      for (int uv = 0; uv < 2; ++uv) {
        const uint64_t full = (uint64_t)uv | ((uint64_t)b << 1); /* union assignment, bit i = uni[i] */
        cx prod = 1.0;
        for (int a = 0; a < ns; ++a) {
          const otensor* T = &pool[sel[a]];
          uint64_t idx = 0;
          for (int i = 0; i < T->rank; ++i) idx |= ((full >> pos[a][i]) & 1ull) << i;
          prod = (a == 0) ? T->val[idx] : prod * T->val[idx];
        }
        term[uv] = prod;
      }
      res[b] = term[0] + term[1];
    }
    cnt->cmul += (double)(ns - 1) * (double)(2 * nout);
    cnt->cadd += (double)nout;
    for (int a = 0; a < ns; ++a) free(pos[a]);
    free(pos);
    /* drop the bucket from the pool (keep the others in order) and add the result */
    int w = 0;
    for (int i = 0, a = 0; i < np; ++i) {
      if (a < ns && sel[a] == i) { free(pool[i].vars); free(pool[i].val); ++a; continue; }
      pool[w++] = pool[i];
    }
    np = w;
    if (ro == 0) {
      acc *= res[0];
      free(res);
      free(uni);
    } else {
      otensor R;
      R.rank = ro;
      R.vars = (int*)malloc(sizeof(int) * ro);
      for (int i = 0; i < ro; ++i) R.vars[i] = uni[i + 1];
      R.val = res;
      pool[np++] = R;
      free(uni);
    }
    free(sel);
  }
  int left = np;
  for (int i = 0; i < np; ++i) { free(pool[i].vars); free(pool[i].val); }
  free(pool);
  free(fixed);
  if (left) return 3; /* a tensor kept a variable outside the order */
  *out = acc;
  return 0;
}

static int key_to_var(const onet* N, int q, int seg) {
  for (int v = 0; v < N->n_vars; ++v)
    if (N->var_qubit[v] == q && N->var_seg[v] == seg) return v;
  return -1;
}

/*
 * Sliced contraction. order_q/order_seg: the elimination order as (qubit,
 * segment) keys of the free non-sliced variables (n_order entries; n_order < 0
 * asks the oracle for its own min-degree order). mu_q/mu_seg: the p sliced
 * variables. Slices s in [s_begin, s_end) are contracted one after another and
 * summed in increasing s (Eq. 5). slice_out (2 doubles per slice) may be NULL.
 * counts (2 doubles: complex multiplications, complex additions) may be NULL.
 */
int orc_contract(int n, size_t n_gates, const int* kind, const int* q0, const int* q1,
                 const double* mats, const uint8_t* bits, const int* order_q,
                 const int* order_seg, int n_order, const int* mu_q, const int* mu_seg, int p,
                 uint64_t s_begin, uint64_t s_end, double* sum_out, double* slice_out,
                 double* counts) {
  if (p < 0 || p > 62 || s_begin > s_end || s_end > (1ull << p)) return -4;
  onet* N = build_net(n, n_gates, kind, q0, q1, mats);
  if (!N) return -1;
  int* mu = (int*)malloc(sizeof(int) * (p ? p : 1));
  for (int j = 0; j < p; ++j) {
    mu[j] = key_to_var(N, mu_q[j], mu_seg[j]);
    if (mu[j] < 0 || N->is_input[mu[j]] || N->is_output[mu[j]]) { free(mu); free_net(N); return -2; }
  }
  int* order = NULL;
  int no = n_order;
  if (n_order >= 0) {
    order = (int*)malloc(sizeof(int) * (no ? no : 1));
    for (int i = 0; i < no; ++i) {
      order[i] = key_to_var(N, order_q[i], order_seg[i]);
      if (order[i] < 0) { free(order); free(mu); free_net(N); return -3; }
    }
  } else {
    /* own order: repeatedly take the free, non-sliced variable with fewest
     * distinct neighbours in the current elimination graph (ties: lowest id) */
    int nv = N->n_vars;
    uint8_t* adj = (uint8_t*)calloc((size_t)nv * nv, 1);
    uint8_t* alive = (uint8_t*)calloc(nv, 1);
    for (int v = 0; v < nv; ++v) alive[v] = !(N->is_input[v] || N->is_output[v]);
    for (int j = 0; j < p; ++j) alive[mu[j]] = 0;
    for (int i = 0; i < N->n_tensors; ++i)
      for (int a = 0; a < N->t[i].rank; ++a)
        for (int b = 0; b < N->t[i].rank; ++b) {
          int x = N->t[i].vars[a], y = N->t[i].vars[b];
          if (x != y) adj[(size_t)x * nv + y] = 1;
        }
    no = 0;
    for (int v = 0; v < nv; ++v) no += alive[v];
    order = (int*)malloc(sizeof(int) * (no ? no : 1));
    for (int step = 0; step < no; ++step) {
      int best = -1, bd = 1 << 30;
      for (int v = 0; v < nv; ++v) {
        if (!alive[v]) continue;
        int d = 0;
        for (int w = 0; w < nv; ++w) d += alive[w] && adj[(size_t)v * nv + w];
        if (d < bd) { bd = d; best = v; }
      }
      order[step] = best;
      alive[best] = 0;
      for (int a = 0; a < nv; ++a) {
        if (!alive[a] || !adj[(size_t)best * nv + a]) continue;
        for (int b = 0; b < nv; ++b)
          if (b != a && alive[b] && adj[(size_t)best * nv + b]) adj[(size_t)a * nv + b] = 1;
      }
    }
    free(adj);
    free(alive);
  }
  ocount cnt = {0, 0};
  cx total = 0.0;
  int rc = 0;
  for (uint64_t s = s_begin; s < s_end; ++s) {
    cx v;
    rc = contract_slice(N, bits, order, no, mu, p, s, &v, &cnt);
    if (rc) break;
    if (slice_out) { slice_out[2 * (s - s_begin)] = creal(v); slice_out[2 * (s - s_begin) + 1] = cimag(v); }
    total += v;
  }
  sum_out[0] = creal(total);
  sum_out[1] = cimag(total);
  if (counts) { counts[0] = cnt.cmul; counts[1] = cnt.cadd; }
  free(order);
  free(mu);
  free_net(N);
  return rc;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
