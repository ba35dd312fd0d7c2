/*
 * tsgne_oracle.c -- plain, slow FP64 CPU reference of the t-SGNE layout loop.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product (the CUDA library and its
 * Python binding) links, loads or calls this file; only the tests, the smoke
 * check and the benchmark's CPU-baseline leg do.  It shares no code with the
 * GPU path.
 *
 * Everything is written as the definitions read, in double precision, with
 * plain loops and no blocking, fusion or reordering.  Section / equation
 * numbers refer to "Efficiently Visualizing Large Graphs" (Li, Xiao, Zhou,
 * arXiv 2310.11186):
 *
 *   tsgo_structure      neighbour graph G_knn,G of Eq. 7 with the graph's own
 *                       edges as neighbours (Sec. 2.2); undirected (Sec. 2)
 *   tsgo_cond_affinity  p_{j|i} of Eq. 2 restricted to N(i), sigma_i by the
 *                       perplexity binary search of Sec. 2.1
 *   tsgo_joint_P        p_ij of Eq. 3, normalised by the total so sum P = 1
 *   tsgo_Z              denominator of Eq. 4 (ordered pairs k != l)
 *   tsgo_kl             objective of Eq. 5
 *   tsgo_gradient       derivative of Eq. 5 w.r.t. y_i (not printed in the
 *                       paper; derived and pinned by finite differences)
 *   tsgo_repulsion_rows per-row repulsive sums, for sampled checks at size
 *   tsgo_optimize       gradient descent with gains, momentum and early
 *                       exaggeration (the paper gives no schedule; the
 *                       published t-SNE defaults are used)
 *   tsgo_shortest_path  ShortestPath graph embedding (Sec. 2.3, Eq. 8): BFS
 *                       distances to d target nodes, capped at l0 + 1
 *   tsgo_bfs_knn        the k nearest neighbours of Eq. 7, found by a k-step
 *                       breadth-first search (Sec. 2.2), before symmetrisation
 *   tsgo_repulsion_tree tree-code approximation of the repulsive sums and Z
 *                       (an extension; the paper sums Eq. 4 exactly); its
 *                       steps are listed above the function
 *   tsgo_repulsion_tree_bounds  tsgo_repulsion_tree plus, per row, a bound on
 *                       its distance from the exact sums (second-order
 *                       remainder of the monopole expansion, derived above
 *                       the function)
 *   tsgo_gradient_tree  tsgo_gradient with the tree code's F^r and Z
 *   tsgo_gradient_rows  tsgo_gradient for listed rows and a given Z (sampled
 *                       checks at sizes where Z is summed separately)
 *
 * Readings of the paper where it is silent (also listed in the design notes):
 *   - N(i) is the set of graph neighbours (k = graph edges), union of both
 *     directions, no self loops, sorted by id.
 *   - the Eq. 2 denominator runs over j in N(i) only;
 *   - if |N(i)| <= perplexity the target entropy ln(perp) is unreachable and
 *     the row is uniform, p_{j|i} = 1/|N(i)| ("saturated row");
 *   - otherwise beta = 1/(2 sigma^2) is bisected from beta = 1 (doubling /
 *     halving while unbounded, midpoints once bracketed) until
 *     |H - ln perp| <= tol or max_iter evaluations; p is taken at the last
 *     evaluated beta; distances are shifted by the row minimum first;
 *   - Eq. 3's 2n is the total T = sum_ij (p_{j|i} + p_{i|j}), which equals 2n
 *     when no node is isolated and keeps sum P = 1 otherwise.
 *
 * Status codes: 0 ok, -1 invalid argument, -2 malformed CSR, -3 out of memory.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define TSGO_OK 0
#define TSGO_EINVAL -1
#define TSGO_EBADCSR -2
#define TSGO_ENOMEM -3

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

/* Checks a CSR: row_ptr[0] = 0, non-decreasing, cols in [0, n). */
int tsgo_check_csr(int32_t n, const int64_t* rp, const int32_t* col) {
  if (n < 0) return TSGO_EINVAL;
  if (rp[0] != 0) return TSGO_EBADCSR;
  for (int32_t i = 0; i < n; ++i)
    if (rp[i + 1] < rp[i]) return TSGO_EBADCSR;
  for (int64_t e = 0; e < rp[n]; ++e)
    if (col[e] < 0 || col[e] >= n) return TSGO_EBADCSR;
  return TSGO_OK;
}

/*
 * Neighbour structure (Eq. 7, neighbours = graph edges, Sec. 2.2).
 * N(i) = { j != i : (i,j) or (j,i) is an input entry }, each row sorted and
 * unique.  Writes out_rp[n+1]; out_col must hold 2*row_ptr[n] entries.
 * Returns nnz (>= 0) or a negative status.
 */
int64_t tsgo_structure(int32_t n, const int64_t* rp, const int32_t* col, int64_t* out_rp, int32_t* out_col) {
  int st = tsgo_check_csr(n, rp, col);
  if (st != TSGO_OK) return st;
  int64_t m = rp[n];
  int64_t* cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  int64_t* cur = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  int32_t* raw = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * m + 1));
  if (!cnt || !cur || !raw) {
    free(cnt); free(cur); free(raw);
    return TSGO_ENOMEM;
  }
  /* both directions of every entry, self loops dropped */
  for (int32_t i = 0; i < n; ++i)
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
      int32_t j = col[e];
      if (j == i) continue;
      cnt[i + 1]++;
      cnt[j + 1]++;
    }
  for (int32_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
  for (int32_t i = 0; i < n; ++i) cur[i] = cnt[i];
  for (int32_t i = 0; i < n; ++i)
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
      int32_t j = col[e];
      if (j == i) continue;
      raw[cur[i]++] = j;
      raw[cur[j]++] = i;
    }
  /* sort each row, drop repeats */
  int64_t nnz = 0;
  out_rp[0] = 0;
  for (int32_t i = 0; i < n; ++i) {
    int64_t a = cnt[i], b = cnt[i + 1];
    qsort(raw + a, (size_t)(b - a), sizeof(int32_t), cmp_i32);
    for (int64_t e = a; e < b; ++e)
      if (e == a || raw[e] != raw[e - 1]) out_col[nnz++] = raw[e];
    out_rp[i + 1] = nnz;
  }
  free(cnt); free(cur); free(raw);
  return nnz;
}

/* Position of column j in sorted row i, or -1. */
static int64_t find_in_row(const int64_t* rp, const int32_t* col, int32_t i, int32_t j) {
  int64_t lo = rp[i], hi = rp[i + 1] - 1;
  while (lo <= hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (col[mid] == j) return mid;
    if (col[mid] < j) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

/* Position of (j,i) for every entry e = (i,j) of a symmetric structure. */
int tsgo_transpose_slots(int32_t n, const int64_t* rp, const int32_t* col, int64_t* tslot) {
  for (int32_t i = 0; i < n; ++i)
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
      int64_t t = find_in_row(rp, col, col[e], i);
      if (t < 0) return TSGO_EBADCSR;
      tslot[e] = t;
    }
  return TSGO_OK;
}

/*
 * Conditional affinities p_{j|i} (Eq. 2 over j in N(i)) with sigma_i from the
 * perplexity binary search (Sec. 2.1): Perp = 2^{H in bits}, i.e. the target
 * entropy in nats is ln(perp).
 *
 * X is n x d row-major FP64.  Writes pcond[nnz] and beta[n] (beta_i =
 * 1/(2 sigma_i^2); 0 for saturated rows and isolated nodes) and, if iters is
 * not NULL, the number of entropy evaluations per row.
 */
int tsgo_cond_affinity(int32_t n, const int64_t* rp, const int32_t* col, const double* X, int32_t d,
                       double perp, double tol, int32_t max_iter, double* pcond, double* beta_out,
                       int32_t* iters) {
  if (n < 0 || d < 1 || !(perp > 1.0) || max_iter < 1) return TSGO_EINVAL;
  const double Hstar = log(perp);
  for (int32_t i = 0; i < n; ++i) {
    int64_t a = rp[i], b = rp[i + 1];
    int64_t k = b - a;
    if (iters) iters[i] = 0;
    beta_out[i] = 0.0;
    if (k == 0) continue;
    /* squared Euclidean distances in R^d */
    double* dist = (double*)malloc(sizeof(double) * (size_t)k);
    if (!dist) return TSGO_ENOMEM;
    for (int64_t e = a; e < b; ++e) {
      const double* xi = X + (int64_t)i * d;
      const double* xj = X + (int64_t)col[e] * d;
      double s = 0.0;
      for (int32_t c = 0; c < d; ++c) {
        double t = xi[c] - xj[c];
        s += t * t;
      }
      dist[e - a] = s;
    }
    if ((double)k <= perp) {
      /* saturated: ln k <= ln perp cannot be reached from above */
      for (int64_t e = a; e < b; ++e) pcond[e] = 1.0 / (double)k;
      free(dist);
      continue;
    }
    double dmin = dist[0];
    for (int64_t t = 1; t < k; ++t)
      if (dist[t] < dmin) dmin = dist[t];
    double beta = 1.0, lo = -INFINITY, hi = INFINITY;
    double S = 0.0;
    int32_t it;
    for (it = 0; it < max_iter; ++it) {
      /* entropy of the row at this beta: H = ln S + beta * E_p[d - dmin] */
      S = 0.0;
      double E = 0.0;
      for (int64_t t = 0; t < k; ++t) {
        double w = exp(-beta * (dist[t] - dmin));
        S += w;
        E += (dist[t] - dmin) * w;
      }
      double H = log(S) + beta * E / S;
      if (fabs(H - Hstar) <= tol || it == max_iter - 1) break;
      if (H > Hstar) {
        lo = beta;
        beta = isinf(hi) ? 2.0 * beta : 0.5 * (beta + hi);
      } else {
        hi = beta;
        beta = isinf(lo) ? 0.5 * beta : 0.5 * (beta + lo);
      }
    }
    if (iters) iters[i] = it + 1;
    beta_out[i] = beta;
    for (int64_t t = 0; t < k; ++t) pcond[a + t] = exp(-beta * (dist[t] - dmin)) / S;
    free(dist);
  }
  return TSGO_OK;
}

/*
 * Joint affinities (Eq. 3): p_ij = (p_{j|i} + p_{i|j}) / T on the symmetric
 * structure, T = sum over all entries of the numerator.  Returns T via *total.
 */
int tsgo_joint_P(int32_t n, const int64_t* rp, const int32_t* col, const double* pcond, double* P,
                 double* total) {
  double T = 0.0;
  for (int32_t i = 0; i < n; ++i)
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
      int64_t t = find_in_row(rp, col, col[e], i);
      if (t < 0) return TSGO_EBADCSR;
      P[e] = pcond[e] + pcond[t];
      T += P[e];
    }
  if (total) *total = T;
  if (T > 0.0)
    for (int64_t e = 0; e < rp[n]; ++e) P[e] /= T;
  return TSGO_OK;
}

/* Student-t kernel w = (1 + ||y_i - y_j||^2)^-1 (Eq. 4 numerator). */
static double kernel_w(const double* Y, int64_t i, int64_t j) {
  double dx = Y[2 * i] - Y[2 * j];
  double dy = Y[2 * i + 1] - Y[2 * j + 1];
  return 1.0 / (1.0 + dx * dx + dy * dy);
}

/* Eq. 4 denominator: Z = sum_k sum_{l != k} w_kl over ordered pairs. */
double tsgo_Z(int32_t n, const double* Y) {
  double Z = 0.0;
  for (int64_t k = 0; k < n; ++k)
    for (int64_t l = 0; l < n; ++l)
      if (l != k) Z += kernel_w(Y, k, l);
  return Z;
}

/*
 * Eq. 5: KL(P || Q) = sum_ij p_ij log(p_ij / q_ij), q_ij = w_ij / Z.
 * Only entries with p_ij > 0 contribute (0 log 0 = 0).
 */
double tsgo_kl(int32_t n, const int64_t* rp, const int32_t* col, const double* P, const double* Y,
               double* Z_out) {
  double Z = tsgo_Z(n, Y);
  double kl = 0.0;
  for (int32_t i = 0; i < n; ++i)
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
      if (!(P[e] > 0.0)) continue;
      double q = kernel_w(Y, i, col[e]) / Z;
      kl += P[e] * log(P[e] / q);
    }
  if (Z_out) *Z_out = Z;
  return kl;
}

/*
 * Gradient of Eq. 5 with the affinities multiplied by alpha (early
 * exaggeration; alpha = 1 is the plain KL gradient):
 *   g_i = 4 * sum_j (alpha p_ij - q_ij) w_ij (y_i - y_j)
 *       = 4 * [ alpha sum_{j in N(i)} p_ij w_ij (y_i - y_j)
 *               - (1/Z) sum_{j != i} w_ij^2 (y_i - y_j) ].
 * G is n x 2.  Returns Z via *Z_out.
 */
int tsgo_gradient(int32_t n, const int64_t* rp, const int32_t* col, const double* P, const double* Y,
                  double alpha, double* G, double* Z_out) {
  double Z = tsgo_Z(n, Y);
  for (int64_t i = 0; i < n; ++i) {
    double ax = 0.0, ay = 0.0, rx = 0.0, ry = 0.0;
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
      int64_t j = col[e];
      double w = kernel_w(Y, i, j);
      ax += P[e] * w * (Y[2 * i] - Y[2 * j]);
      ay += P[e] * w * (Y[2 * i + 1] - Y[2 * j + 1]);
    }
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      double w = kernel_w(Y, i, j);
      rx += w * w * (Y[2 * i] - Y[2 * j]);
      ry += w * w * (Y[2 * i + 1] - Y[2 * j + 1]);
    }
    G[2 * i] = 4.0 * (alpha * ax - rx / Z);
    G[2 * i + 1] = 4.0 * (alpha * ay - ry / Z);
  }
  if (Z_out) *Z_out = Z;
  return TSGO_OK;
}

/*
 * Rows [i0, i1): F_rep_i = sum_{j != i} w_ij^2 (y_i - y_j) (n x 2 slots i0..i1-1
 * of Frep) and zrow_i = sum_{j != i} w_ij, so that Z = sum_i zrow_i.  Lets a
 * caller split the quadratic work over threads or check sampled rows.
 */
int tsgo_repulsion_rows(int32_t n, const double* Y, int32_t i0, int32_t i1, double* Frep, double* zrow) {
  if (i0 < 0 || i1 > n || i0 > i1) return TSGO_EINVAL;
  for (int64_t i = i0; i < i1; ++i) {
    double rx = 0.0, ry = 0.0, z = 0.0;
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      double w = kernel_w(Y, i, j);
      z += w;
      rx += w * w * (Y[2 * i] - Y[2 * j]);
      ry += w * w * (Y[2 * i + 1] - Y[2 * j + 1]);
    }
    Frep[2 * (i - i0)] = rx;
    Frep[2 * (i - i0) + 1] = ry;
    zrow[i - i0] = z;
  }
  return TSGO_OK;
}

/* Attractive sums F_attr_i = sum_{j in N(i)} p_ij w_ij (y_i - y_j) for listed rows. */
int tsgo_attraction_rows(int32_t n, const int64_t* rp, const int32_t* col, const double* P, const double* Y,
                         const int32_t* rows, int32_t nrows, double* Fattr) {
  for (int32_t r = 0; r < nrows; ++r) {
    int64_t i = rows[r];
    if (i < 0 || i >= n) return TSGO_EINVAL;
    double ax = 0.0, ay = 0.0;
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
      int64_t j = col[e];
      double w = kernel_w(Y, i, j);
      ax += P[e] * w * (Y[2 * i] - Y[2 * j]);
      ay += P[e] * w * (Y[2 * i + 1] - Y[2 * j + 1]);
    }
    Fattr[2 * r] = ax;
    Fattr[2 * r + 1] = ay;
  }
  return TSGO_OK;
}

/*
 * Gradient descent on Eq. 5 (the paper states only that the iteration count
 * is a fixed constant, Sec. 3.3).  Schedule, per iteration t (0-based,
 * counting from t0):
 *   alpha = ee   if t < ee_iters else 1      (early exaggeration)
 *   mu    = mom0 if t < ee_iters else mom1   (momentum)
 *   g = gradient with alpha
 *   per coordinate: gain += 0.2 if g * upd < 0, else gain *= 0.8;
 *                   gain = max(gain, min_gain);
 *                   upd = mu * upd - eta * gain * g;  y += upd
 * Y, upd, gains are n x 2 and updated in place.
 */
int tsgo_optimize(int32_t n, const int64_t* rp, const int32_t* col, const double* P, double* Y, double* upd,
                  double* gains, int32_t t0, int32_t n_iter, double ee, int32_t ee_iters, double mom0,
                  double mom1, double eta, double min_gain) {
  double* G = (double*)malloc(sizeof(double) * 2 * (size_t)(n > 0 ? n : 1));
  if (!G) return TSGO_ENOMEM;
  for (int32_t t = t0; t < t0 + n_iter; ++t) {
    double alpha = t < ee_iters ? ee : 1.0;
    double mu = t < ee_iters ? mom0 : mom1;
    tsgo_gradient(n, rp, col, P, Y, alpha, G, NULL);
    for (int64_t c = 0; c < 2 * (int64_t)n; ++c) {
      if (G[c] * upd[c] < 0.0)
        gains[c] += 0.2;
      else
        gains[c] *= 0.8;
      if (gains[c] < min_gain) gains[c] = min_gain;
      upd[c] = mu * upd[c] - eta * gains[c] * G[c];
      Y[c] += upd[c];
    }
  }
  free(G);
  return TSGO_OK;
}

/*
 * ShortestPath embedding (Sec. 2.3, Eq. 8): E_it = dist(v_i, target_t) when
 * that distance is <= l0, else l0 + 1 (also when no path exists).  One BFS
 * per target over the undirected graph given by a symmetric CSR.  X is n x d
 * row-major (FP64 here; the values are small integers).
 */
int tsgo_shortest_path(int32_t n, const int64_t* rp, const int32_t* col, const int32_t* targets, int32_t d,
                       int32_t l0, double* X) {
  if (n < 1 || d < 1 || l0 < 0) return TSGO_EINVAL;
  int32_t* dist = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  if (!dist || !queue) {
    free(dist); free(queue);
    return TSGO_ENOMEM;
  }
  for (int32_t t = 0; t < d; ++t) {
    int32_t s = targets[t];
    if (s < 0 || s >= n) {
      free(dist); free(queue);
      return TSGO_EINVAL;
    }
    for (int32_t i = 0; i < n; ++i) dist[i] = -1;
    int32_t head = 0, tail = 0;
    dist[s] = 0;
    queue[tail++] = s;
    while (head < tail) {
      int32_t v = queue[head++];
      for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
        int32_t w = col[e];
        if (dist[w] < 0) {
          dist[w] = dist[v] + 1;
          queue[tail++] = w;
        }
      }
    }
    for (int32_t i = 0; i < n; ++i)
      X[(int64_t)i * d + t] = (dist[i] >= 0 && dist[i] <= l0) ? (double)dist[i] : (double)(l0 + 1);
  }
  free(dist);
  free(queue);
  return TSGO_OK;
}

/*
 * k nearest neighbours of every node by breadth-first search on G (Eq. 7,
 * Sec. 2.2): the first k nodes other than i in BFS order from i, levels in
 * order, and within a level in order of discovery, each node's neighbours
 * scanned in ascending id (rows of rp/col must be sorted); fewer when i's
 * component is smaller.  out is n x k (row i: its list in BFS order), cnt[i]
 * its length.  The caller symmetrises the lists by union.
 */
int tsgo_bfs_knn(int32_t n, const int64_t* rp, const int32_t* col, int32_t k, int32_t* out, int32_t* cnt) {
  if (n < 1 || k < 1) return TSGO_EINVAL;
  char* seen = (char*)calloc((size_t)n, 1);
  int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  if (!seen || !queue) {
    free(seen); free(queue);
    return TSGO_ENOMEM;
  }
  for (int32_t i = 0; i < n; ++i) {
    int32_t head = 0, tail = 0, found = 0;
    queue[tail++] = i;
    seen[i] = 1;
    while (head < tail && found < k) {
      int32_t v = queue[head++];
      for (int64_t e = rp[v]; e < rp[v + 1] && found < k; ++e) {
        int32_t w = col[e];
        if (seen[w]) continue;
        seen[w] = 1;
        queue[tail++] = w;
        out[(int64_t)i * k + found++] = w;
      }
    }
    cnt[i] = found;
    for (int32_t t = 0; t < tail; ++t) seen[queue[t]] = 0;
  }
  free(seen);
  free(queue);
  return TSGO_OK;
}

/*
 * ---------------------------------------------------------------------------
 * Tree-code approximation of the repulsive sums (an extension: the paper
 * evaluates the O(|V|^2) sum of Eq. 4 exactly, Sec. 2.1 "Time complexity").
 * The approximation is defined by the steps below; decisions that pick
 * interactions (cell codes, tree shape, acceptance) are taken in FP32, as the
 * GPU takes them, and the sums are then accumulated in FP64.
 *
 *  1. Bounding square (FP32): lo = (min x, min y), side = max(max x - min x,
 *     max y - min y) floored at 1e-30; scale = 2^32 / side in FP64.
 *  2. Cell of a point per axis, in FP64: c = (v - lo) * scale, truncated to
 *     an integer and clamped to [0, 2^32 - 1] (NaN -> 0); key = 64-bit
 *     Morton interleave of the two cells, x in the even bits.  32 bits per
 *     axis keep points apart even when a few outliers stretch the square
 *     to thousands of times the bulk's size.
 *  3. Order: points sorted by (key, index).  Position k of the sorted order
 *     gets the 96-bit augmented key (key, k), unique per point.
 *  4. Tree: the binary radix tree of the augmented keys.  A node covers
 *     sorted positions [f, l]; if f < l it splits at the highest bit in which
 *     the augmented keys of f and l differ: the left child holds the
 *     positions whose bit is 0.  A single position is a leaf.
 *  5. Node summaries (FP32): count; coordinate sums, left + right; bounding
 *     box; centre = sums / count; r2 = (longest box side)^2.
 *  6. Groups: the maximal subtrees of at most 32 points (nodes of <= 32
 *     points whose parent has more; the root if n <= 32), in sorted order.
 *     They partition the sorted positions into runs, each a Morton cell;
 *     a group's box is the bounding box of its points.
 *  7. Walk, per group, from the root, left child before right:
 *     - a leaf is an exact interaction with its point;
 *     - otherwise d2 = squared distance from the node's centre to the group
 *       box (0 inside); if r2 < theta^2 * d2 the node is one interaction of
 *       weight count at its centre;
 *     - otherwise, if count <= bucket, exact interactions with each of its
 *       points; else both children are walked.
 *     An exact interaction of point i with point j != i adds w = 1/(1 + |y_i
 *     - y_j|^2) to zrow_i and w^2 (y_i - y_j) to F_i; a node interaction
 *     adds count * w and count * w^2 (y_i - c) with w taken at the centre c.
 *     A point never interacts with itself exactly.
 *  Z = sum_i zrow_i.  theta = 0 accepts no node and reduces to the exact sums
 *  of tsgo_repulsion_rows.
 * ---------------------------------------------------------------------------
 */
typedef struct {
  int32_t first, last, left, right; /* left/right: node ids, -1 for a leaf */
  float sx, sy, x0, y0, x1, y1, cx, cy, r2;
  /* For the error bound only (FP64, from the node's points; no effect on
   * the sums): s2 = sum_j |c - y_j|^2 about the FP32 centre c; cerr = |c -
   * mean|, the rounding of the FP32 centre; a = largest distance from c to a
   * corner of the box, which bounds |c - y_j|. */
  double s2, cerr, a;
} tsgo_tnode;

typedef struct {
  uint64_t key;
  int32_t idx;
} tsgo_keyed;

static int cmp_keyed(const void* a, const void* b) {
  const tsgo_keyed* x = (const tsgo_keyed*)a;
  const tsgo_keyed* y = (const tsgo_keyed*)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  return (x->idx > y->idx) - (x->idx < y->idx);
}

static uint64_t spread_bits32(uint32_t v) {
  uint64_t r = 0;
  for (int b = 0; b < 32; ++b) r |= (uint64_t)((v >> b) & 1u) << (2 * b);
  return r;
}

static uint32_t cell32(float v, double lo, double scale) {
  double c = ((double)v - lo) * scale;
  if (!(c >= 0.0)) return 0u;
  if (c >= 4294967295.0) return 4294967295u;
  return (uint32_t)c;
}

/* Bit b of the augmented key (key, pos): b in [32, 96) is key bit b - 32,
 * b in [0, 32) is position bit b. */
static int aug_bit(uint64_t key, uint32_t pos, int b) {
  return b >= 32 ? (int)((key >> (b - 32)) & 1u) : (int)((pos >> b) & 1u);
}

/* Moments of an internal node's points about its FP32 centre (bound only). */
static void node_moments(tsgo_tnode* t, const float* xs, const float* ys) {
  double mx = 0.0, my = 0.0, s2 = 0.0;
  const double m = (double)(t->last - t->first + 1);
  for (int32_t k = t->first; k <= t->last; ++k) {
    mx += xs[k];
    my += ys[k];
  }
  mx /= m;
  my /= m;
  for (int32_t k = t->first; k <= t->last; ++k) {
    const double dx = (double)t->cx - xs[k], dy = (double)t->cy - ys[k];
    s2 += dx * dx + dy * dy;
  }
  t->s2 = s2;
  t->cerr = hypot((double)t->cx - mx, (double)t->cy - my);
  double a2 = 0.0;
  const float bx[2] = {t->x0, t->x1}, by[2] = {t->y0, t->y1};
  for (int p = 0; p < 2; ++p)
    for (int q = 0; q < 2; ++q) {
      const double dx = (double)t->cx - bx[p], dy = (double)t->cy - by[q];
      if (dx * dx + dy * dy > a2) a2 = dx * dx + dy * dy;
    }
  t->a = sqrt(a2);
}

/* Builds the subtree over sorted positions [f, l]; returns its node id. */
static int32_t tree_build(const uint64_t* keys, const float* xs, const float* ys, int32_t f, int32_t l,
                          tsgo_tnode* nodes, int32_t* count) {
  int32_t id = (*count)++;
  tsgo_tnode* t = &nodes[id];
  t->first = f;
  t->last = l;
  if (f == l) {
    t->left = t->right = -1;
    t->sx = t->x0 = t->x1 = t->cx = xs[f];
    t->sy = t->y0 = t->y1 = t->cy = ys[f];
    t->r2 = 0.0f;
    t->s2 = t->cerr = t->a = 0.0;
    return id;
  }
  int bit = 95;
  while (aug_bit(keys[f], (uint32_t)f, bit) == aug_bit(keys[l], (uint32_t)l, bit)) --bit;
  int32_t g = f;
  while (g + 1 <= l && aug_bit(keys[g + 1], (uint32_t)(g + 1), bit) == 0) ++g;
  int32_t L = tree_build(keys, xs, ys, f, g, nodes, count);
  int32_t R = tree_build(keys, xs, ys, g + 1, l, nodes, count);
  t = &nodes[id];
  const tsgo_tnode* a = &nodes[L];
  const tsgo_tnode* b = &nodes[R];
  t->left = L;
  t->right = R;
  t->sx = a->sx + b->sx;
  t->sy = a->sy + b->sy;
  t->x0 = fminf(a->x0, b->x0);
  t->y0 = fminf(a->y0, b->y0);
  t->x1 = fmaxf(a->x1, b->x1);
  t->y1 = fmaxf(a->y1, b->y1);
  float cnt = (float)(l - f + 1);
  t->cx = t->sx / cnt;
  t->cy = t->sy / cnt;
  float r = fmaxf(t->x1 - t->x0, t->y1 - t->y0);
  t->r2 = r * r;
  node_moments(t, xs, ys);
  return id;
}

/*
 * Error bound of one accepted node (used by tsgo_repulsion_tree_bounds).
 *
 * A node of m points y_j with centre c stands for the m exact terms
 * f(y_i - y_j) by m f(y_i - c), for f = w (the Z row) and f = w^2 u (the
 * force), w(u) = 1 / (1 + |u|^2).  Write y_i - y_j = u + delta_j with
 * u = y_i - c and delta_j = c - y_j.  Taylor's theorem with the integral
 * remainder along the segment from u to u + delta_j gives
 *   f(u + delta_j) = f(u) + Df(u)[delta_j] + R_j,
 *   |R_j| <= 1/2 |delta_j|^2 sup_{t in [0,1]} ||D^2 f(u + t delta_j)||.
 * Summed over the node, the first-order terms add up to m Df(u)[c - mean],
 * which vanishes when c is the mean of the points (the node's centre is
 * their coordinate sum over the count, so only its FP32 rounding remains),
 * and every point of the segment lies at distance >= rho = max(|u| - a, 0)
 * from the origin, a >= |delta_j| being the largest distance from c to a
 * corner of the node's box.  Hence
 *   |sum_j f(y_i - y_j) - m f(u)| <= m ||Df(u)|| |c - mean|
 *                                    + 1/2 (sum_j |delta_j|^2) G_f(rho),
 * with G_f(rho) = sup_{|x| >= rho} ||D^2 f(x)|| (operator norm on unit
 * directions).  The derivatives, with s = |x|^2:
 *   w:      Dw = -2 w^2 x, so ||Dw|| = 2 |x| w^2;
 *           D^2 w = -2 w^2 I + 8 w^3 x x^T, eigenvalues -2 w^2 and
 *           2 w^3 (3 s - 1), so ||D^2 w|| = 2 w^2 for s <= 1 and
 *           2 w^3 (3 s - 1) for s > 1 -- non-increasing in |x|, so G_w(rho)
 *           is its value at rho;
 *   w^2 x:  D[h] = w^2 h - 4 w^3 (x.h) x, eigenvalues w^2 and w^2 (1 - 3 s) /
 *           (1 + s), so ||D|| = w^2 max(1, |1 - 3 s| / (1 + s));
 *           D^2[h, h] = 24 w^4 (x.h)^2 x - 4 w^3 x - 8 w^3 (x.h) h for |h| = 1,
 *           of norm <= 12 w^3 |x| + 24 w^4 |x|^3 = (12 t + 36 t^3) / (1 + t^2)^4
 *           at t = |x|; this rises up to t = 1/sqrt(3) and falls after it, so
 *           G(rho) is its value at max(rho, 1/sqrt(3)).
 * If the node holds point i itself, the monopole also stands for the j = i
 * term that the exact sums leave out: w(0) = 1 in the Z row, 0 in the force.
 * The bound is returned in two parts per row: the centre-rounding (first
 * order) part and the remainder (second order) part.
 */
/* Planted mistakes for the tests that show the bound check catches them
 * (0 = none, the default): 1 = a node's count taken one short, 2 = the
 * node's box centre used in place of its centre of mass, 3 = the force of an
 * accepted node with the wrong sign, 4 = a point paired with itself in the
 * exact sums of an opened bucket.  Test infrastructure only. */
static int g_tree_mutation = 0;
void tsgo_tree_mutation(int32_t which) { g_tree_mutation = which; }

static double bound_w_hess(double rho) {
  const double s = rho * rho, w = 1.0 / (1.0 + s);
  return s <= 1.0 ? 2.0 * w * w : 2.0 * w * w * w * (3.0 * s - 1.0);
}

static double bound_f_hess(double rho) {
  double t = rho > 0.57735026918962576 ? rho : 0.57735026918962576;
  const double q = 1.0 + t * t;
  return (12.0 * t + 36.0 * t * t * t) / (q * q * q * q);
}

typedef struct {
  const tsgo_tnode* nodes;
  const float* xs;
  const float* ys;
  int32_t g0, g1; /* group's sorted positions [g0, g1) */
  float bx0, by0, bx1, by1, theta2;
  int32_t bucket;
  double* F;    /* per sorted position */
  double* zrow; /* per sorted position */
  double* bnd;  /* NULL, or per sorted position: Z first / second order, F first / second order */
} tsgo_walk;

static void node_bound(const tsgo_walk* w, const tsgo_tnode* t, int32_t i) {
  const double m = (double)(t->last - t->first + 1);
  const double ux = (double)w->xs[i] - (double)t->cx, uy = (double)w->ys[i] - (double)t->cy;
  const double s = ux * ux + uy * uy, D = sqrt(s), k = 1.0 / (1.0 + s);
  double rho = D - t->a;
  if (rho < 0.0) rho = 0.0;
  double* b = w->bnd + 4 * (size_t)i;
  const double lin_f = fabs(1.0 - 3.0 * s) / (1.0 + s);
  b[0] += m * 2.0 * D * k * k * t->cerr;
  b[1] += 0.5 * t->s2 * bound_w_hess(rho) + ((i >= t->first && i <= t->last) ? 1.0 : 0.0);
  b[2] += m * k * k * (lin_f > 1.0 ? lin_f : 1.0) * t->cerr;
  b[3] += 0.5 * t->s2 * bound_f_hess(rho);
}

static void exact_pairs(const tsgo_walk* w, int32_t j) {
  for (int32_t i = w->g0; i < w->g1; ++i) {
    if (i == j) continue;
    double dx = (double)w->xs[i] - (double)w->xs[j];
    double dy = (double)w->ys[i] - (double)w->ys[j];
    double k = 1.0 / (1.0 + dx * dx + dy * dy);
    w->zrow[i] += k;
    w->F[2 * i] += k * k * dx;
    w->F[2 * i + 1] += k * k * dy;
  }
}

static void tree_walk(const tsgo_walk* w, int32_t id) {
  const tsgo_tnode* t = &w->nodes[id];
  if (t->left < 0) {
    exact_pairs(w, t->first);
    return;
  }
  float dx = fmaxf(fmaxf(w->bx0 - t->cx, t->cx - w->bx1), 0.0f);
  float dy = fmaxf(fmaxf(w->by0 - t->cy, t->cy - w->by1), 0.0f);
  float d2 = dx * dx + dy * dy;
  if (t->r2 < w->theta2 * d2) {
    double c = (double)(t->last - t->first + 1);
    double mx = t->cx, my = t->cy, sg = 1.0;
    if (g_tree_mutation == 1) c -= 1.0;
    if (g_tree_mutation == 2) {
      mx = 0.5 * ((double)t->x0 + (double)t->x1);
      my = 0.5 * ((double)t->y0 + (double)t->y1);
    }
    if (g_tree_mutation == 3) sg = -1.0;
    for (int32_t i = w->g0; i < w->g1; ++i) {
      if (w->bnd) node_bound(w, t, i);
      double ex = (double)w->xs[i] - mx;
      double ey = (double)w->ys[i] - my;
      double k = 1.0 / (1.0 + ex * ex + ey * ey);
      w->zrow[i] += c * k;
      w->F[2 * i] += sg * c * k * k * ex;
      w->F[2 * i + 1] += sg * c * k * k * ey;
    }
    return;
  }
  if (t->last - t->first + 1 <= w->bucket) {
    for (int32_t j = t->first; j <= t->last; ++j) {
      exact_pairs(w, j);
      if (g_tree_mutation == 4 && j >= w->g0 && j < w->g1) w->zrow[j] += 1.0;
    }
    return;
  }
  tree_walk(w, t->left);
  tree_walk(w, t->right);
}

/* Appends the groups under node id (maximal subtrees of <= 32 points). */
static void collect_groups(const tsgo_tnode* nodes, int32_t id, int32_t* gfirst, int32_t* glast, int32_t* ng) {
  const tsgo_tnode* t = &nodes[id];
  if (t->last - t->first + 1 <= 32) {
    gfirst[*ng] = t->first;
    glast[*ng] = t->last;
    ++*ng;
    return;
  }
  collect_groups(nodes, t->left, gfirst, glast, ng);
  collect_groups(nodes, t->right, gfirst, glast, ng);
}

/*
 * Y: n x 2 layout (FP32 values carried in doubles); theta >= 0; bucket >= 1.
 * Frep (n x 2) and zrow (n) come back in the input order; returns Z through
 * *Z_out.  bnd: NULL, or n x 4 (input order) for tsgo_repulsion_tree_bounds.
 */
static int tree_pass(int32_t n, const double* Y, double theta, int32_t bucket, double* Frep, double* zrow,
                     double* Z_out, double* bnd) {
  if (n < 1 || !(theta >= 0.0) || bucket < 1) return TSGO_EINVAL;
  float* xs = (float*)malloc(sizeof(float) * (size_t)n);
  float* ys = (float*)malloc(sizeof(float) * (size_t)n);
  tsgo_keyed* kv = (tsgo_keyed*)malloc(sizeof(tsgo_keyed) * (size_t)n);
  uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)n);
  tsgo_tnode* nodes = (tsgo_tnode*)malloc(sizeof(tsgo_tnode) * (size_t)(2 * n - 1));
  double* F = (double*)calloc(2 * (size_t)n, sizeof(double));
  double* zr = (double*)calloc((size_t)n, sizeof(double));
  double* bs = bnd ? (double*)calloc(4 * (size_t)n, sizeof(double)) : NULL;
  int32_t* gfirst = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int32_t* glast = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  if (!xs || !ys || !kv || !keys || !nodes || !F || !zr || !gfirst || !glast || (bnd && !bs)) {
    free(xs); free(ys); free(kv); free(keys); free(nodes); free(F); free(zr); free(gfirst); free(glast); free(bs);
    return TSGO_ENOMEM;
  }
  /* 1-2: bounding square and keys */
  float lx = (float)Y[0], ly = (float)Y[1], hx = lx, hy = ly;
  for (int32_t i = 1; i < n; ++i) {
    float x = (float)Y[2 * i], y = (float)Y[2 * i + 1];
    lx = fminf(lx, x);
    hx = fmaxf(hx, x);
    ly = fminf(ly, y);
    hy = fmaxf(hy, y);
  }
  float side = fmaxf(fmaxf(hx - lx, hy - ly), 1e-30f);
  double scale = 4294967296.0 / (double)side;
  for (int32_t i = 0; i < n; ++i) {
    uint32_t cx = cell32((float)Y[2 * i], (double)lx, scale), cy = cell32((float)Y[2 * i + 1], (double)ly, scale);
    kv[i].key = spread_bits32(cx) | (spread_bits32(cy) << 1);
    kv[i].idx = i;
  }
  /* 3: order */
  qsort(kv, (size_t)n, sizeof(tsgo_keyed), cmp_keyed);
  for (int32_t k = 0; k < n; ++k) {
    xs[k] = (float)Y[2 * kv[k].idx];
    ys[k] = (float)Y[2 * kv[k].idx + 1];
    keys[k] = kv[k].key;
  }
  /* 4-5: tree */
  int32_t count = 0;
  int32_t root = tree_build(keys, xs, ys, 0, n - 1, nodes, &count);
  /* 6-7: groups and walks */
  float th = (float)theta;
  tsgo_walk w;
  w.nodes = nodes;
  w.xs = xs;
  w.ys = ys;
  w.theta2 = th * th;
  w.bucket = bucket;
  w.F = F;
  w.zrow = zr;
  w.bnd = bs;
  int32_t ng = 0;
  collect_groups(nodes, root, gfirst, glast, &ng);
  for (int32_t g = 0; g < ng; ++g) {
    int32_t g0 = gfirst[g], g1 = glast[g] + 1;
    w.g0 = g0;
    w.g1 = g1;
    w.bx0 = w.bx1 = xs[g0];
    w.by0 = w.by1 = ys[g0];
    for (int32_t i = g0 + 1; i < g1; ++i) {
      w.bx0 = fminf(w.bx0, xs[i]);
      w.bx1 = fmaxf(w.bx1, xs[i]);
      w.by0 = fminf(w.by0, ys[i]);
      w.by1 = fmaxf(w.by1, ys[i]);
    }
    tree_walk(&w, root);
  }
  double Z = 0.0;
  for (int32_t k = 0; k < n; ++k) {
    int32_t i = kv[k].idx;
    Frep[2 * i] = F[2 * k];
    Frep[2 * i + 1] = F[2 * k + 1];
    if (zrow) zrow[i] = zr[k];
    if (bnd)
      for (int q = 0; q < 4; ++q) bnd[4 * (size_t)i + q] = bs[4 * (size_t)k + q];
    Z += zr[k];
  }
  if (Z_out) *Z_out = Z;
  free(xs); free(ys); free(kv); free(keys); free(nodes); free(F); free(zr); free(gfirst); free(glast); free(bs);
  return TSGO_OK;
}

int tsgo_repulsion_tree(int32_t n, const double* Y, double theta, int32_t bucket, double* Frep, double* zrow,
                        double* Z_out) {
  return tree_pass(n, Y, theta, bucket, Frep, zrow, Z_out, NULL);
}

/*
 * tsgo_repulsion_tree with, per row i (input order), bnd[4 i .. 4 i + 3] =
 * bounds on |zrow_i - exact zrow_i| (centre-rounding part, remainder part)
 * and on |F_i - exact F_i| (Euclidean norm; the same two parts), summed over
 * the nodes the walk accepted for i's group (derivation above node_bound).
 * Rows whose group accepted no node are exact: their bounds are 0.
 */
int tsgo_repulsion_tree_bounds(int32_t n, const double* Y, double theta, int32_t bucket, double* Frep,
                               double* zrow, double* Z_out, double* bnd) {
  if (!bnd) return TSGO_EINVAL;
  return tree_pass(n, Y, theta, bucket, Frep, zrow, Z_out, bnd);
}

/*
 * Gradient of Eq. 5 (as tsgo_gradient) with the repulsive sums and Z taken
 * from the tree code: g_i = 4 (alpha F^a_i - F^r_i / Z).
 */
int tsgo_gradient_tree(int32_t n, const int64_t* rp, const int32_t* col, const double* P, const double* Y,
                       double alpha, double theta, int32_t bucket, double* G, double* Z_out) {
  double* Fr = (double*)malloc(sizeof(double) * 2 * (size_t)(n > 0 ? n : 1));
  if (!Fr) return TSGO_ENOMEM;
  double Z = 0.0;
  int st = tsgo_repulsion_tree(n, Y, theta, bucket, Fr, NULL, &Z);
  if (st != TSGO_OK) {
    free(Fr);
    return st;
  }
  for (int64_t i = 0; i < n; ++i) {
    double ax = 0.0, ay = 0.0;
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
      int64_t j = col[e];
      double w = kernel_w(Y, i, j);
      ax += P[e] * w * (Y[2 * i] - Y[2 * j]);
      ay += P[e] * w * (Y[2 * i + 1] - Y[2 * j + 1]);
    }
    G[2 * i] = 4.0 * (alpha * ax - Fr[2 * i] / Z);
    G[2 * i + 1] = 4.0 * (alpha * ay - Fr[2 * i + 1] / Z);
  }
  free(Fr);
  if (Z_out) *Z_out = Z;
  return TSGO_OK;
}

/*
 * ---------------------------------------------------------------------------
 * Random-walk estimate of p_{j|i} (Sec. 2.1, Eq. 6), on the neighbour graph
 * N of Eq. 7 (the symmetric structure rp, col).
 *
 *  - Transition from u: to v in N(u) with probability proportional to
 *    exp(-||x_u - x_v||^2) (the exponent's sign is read as negative; the
 *    squared distances are shifted by the row minimum before exp, which does
 *    not change the normalised probabilities).  Distances in FP64, summed
 *    over dimensions in index order; the walk takes the first neighbour whose
 *    running sum of weights exceeds U * (total weight), U uniform in [0, 1).
 *    A node without neighbours keeps the walk where it is.
 *  - R walks of L steps start at every node i.  Reading of Eq. 6: a walk
 *    goes "from i to j" when it ends at j; walks ending at i are dropped
 *    (p_ii = 0), so p_{j|i} = count_ij / R.  With L = 1 the expectation of
 *    p_{j|i} is the transition probability itself, i.e. Eq. 2 with
 *    2 sigma^2 = 1.
 *  - U for step s of walk r from node i is the SplitMix64 output number
 *    k = 1 + (i R + r) L + s of the sequence seeded with
 *    seed ^ 0xD1B54A32D192ED03: state = that seed + k * 0x9E3779B97F4A7C15,
 *    mixed as published (xor-shift 30, * 0xBF58476D1CE4E5B9, xor-shift 27,
 *    * 0x94D049BB133111EB, xor-shift 31); U = (output >> 11) * 2^-53.
 *
 * Output: per node i the distinct end points j != i in increasing order with
 * their counts: wrp[0..n], wcol / wcnt of length wrp[n] <= n R.
 * ---------------------------------------------------------------------------
 */
static uint64_t sm64_output(uint64_t seed, uint64_t k) {
  uint64_t z = seed + k * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static double sq_dist(const double* X, int32_t d, int64_t u, int64_t v) {
  double s = 0.0;
  for (int32_t k = 0; k < d; ++k) {
    double t = X[u * d + k] - X[v * d + k];
    s += t * t;
  }
  return s;
}

static int32_t walk_step(const int64_t* rp, const int32_t* col, const double* X, int32_t d, int32_t u, double U) {
  int64_t a = rp[u], b = rp[u + 1];
  if (a == b) return u;
  double dmin = INFINITY;
  for (int64_t e = a; e < b; ++e) {
    double s = sq_dist(X, d, u, col[e]);
    if (s < dmin) dmin = s;
  }
  double total = 0.0;
  for (int64_t e = a; e < b; ++e) total += exp(-(sq_dist(X, d, u, col[e]) - dmin));
  double target = U * total, run = 0.0;
  for (int64_t e = a; e < b; ++e) {
    run += exp(-(sq_dist(X, d, u, col[e]) - dmin));
    if (run > target) return col[e];
  }
  return col[b - 1];
}

int tsgo_random_walk_counts(int32_t n, const int64_t* rp, const int32_t* col, const double* X, int32_t d,
                            int32_t R, int32_t L, uint64_t seed, int64_t* wrp, int32_t* wcol, int32_t* wcnt) {
  if (n < 1 || R < 1 || L < 1 || d < 1) return TSGO_EINVAL;
  int st = tsgo_check_csr(n, rp, col);
  if (st != TSGO_OK) return st;
  const uint64_t s0 = seed ^ 0xD1B54A32D192ED03ull;
  int32_t* ends = (int32_t*)malloc(sizeof(int32_t) * (size_t)R);
  if (!ends) return TSGO_ENOMEM;
  int64_t m = 0;
  wrp[0] = 0;
  for (int32_t i = 0; i < n; ++i) {
    int32_t ne = 0;
    for (int32_t r = 0; r < R; ++r) {
      int32_t u = i;
      for (int32_t s = 0; s < L; ++s) {
        uint64_t k = 1u + ((uint64_t)i * (uint64_t)R + (uint64_t)r) * (uint64_t)L + (uint64_t)s;
        double U = (double)(sm64_output(s0, k) >> 11) * (1.0 / 9007199254740992.0);
        u = walk_step(rp, col, X, d, u, U);
      }
      if (u != i) ends[ne++] = u;
    }
    qsort(ends, (size_t)ne, sizeof(int32_t), cmp_i32);
    for (int32_t t = 0; t < ne;) {
      int32_t u = t;
      while (u < ne && ends[u] == ends[t]) ++u;
      wcol[m] = ends[t];
      wcnt[m] = u - t;
      ++m;
      t = u;
    }
    wrp[i + 1] = m;
  }
  free(ends);
  return TSGO_OK;
}

/*
 * p_{j|i} = count_ij / R on a structure (rp, col) that contains every walk
 * pair (i, j) (e.g. its symmetrisation); 0 where no walk from i ended at j.
 */
int tsgo_random_walk_pcond(int32_t n, const int64_t* wrp, const int32_t* wcol, const int32_t* wcnt, int32_t R,
                           const int64_t* rp, const int32_t* col, double* pcond) {
  for (int32_t i = 0; i < n; ++i)
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
      pcond[e] = 0.0;
      for (int64_t t = wrp[i]; t < wrp[i + 1]; ++t)
        if (wcol[t] == col[e]) pcond[e] = (double)wcnt[t] / (double)R;
    }
  return TSGO_OK;
}

/* Output number k (k >= 1) of the SplitMix64 sequence seeded with seed. */
uint64_t tsgo_splitmix64(uint64_t seed, uint64_t k) { return sm64_output(seed, k); }

/*
 * Gradient rows for a given normaliser Z (for sampled checks at sizes where
 * the O(n^2) Z is computed separately): for each listed row i,
 *   g_i = 4 (alpha sum_{j in N(i)} p_ij w_ij (y_i - y_j)
 *            - (1/Z) sum_{j != i} w_ij^2 (y_i - y_j)).
 * G is nrows x 2 in the order of rows.
 */
int tsgo_gradient_rows(int32_t n, const int64_t* rp, const int32_t* col, const double* P, const double* Y,
                       double alpha, double Z, const int32_t* rows, int32_t nrows, double* G) {
  for (int32_t r = 0; r < nrows; ++r) {
    int64_t i = rows[r];
    if (i < 0 || i >= n) return TSGO_EINVAL;
    double ax = 0.0, ay = 0.0, rx = 0.0, ry = 0.0;
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
      int64_t j = col[e];
      double w = kernel_w(Y, i, j);
      ax += P[e] * w * (Y[2 * i] - Y[2 * j]);
      ay += P[e] * w * (Y[2 * i + 1] - Y[2 * j + 1]);
    }
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      double w = kernel_w(Y, i, j);
      rx += w * w * (Y[2 * i] - Y[2 * j]);
      ry += w * w * (Y[2 * i + 1] - Y[2 * j + 1]);
    }
    G[2 * r] = 4.0 * (alpha * ax - rx / Z);
    G[2 * r + 1] = 4.0 * (alpha * ay - ry / Z);
  }
  return TSGO_OK;
}
