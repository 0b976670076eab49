/*
 * CPU oracle for connected-components labelling of a 2D binary image (and,
 * at the end of the file, of a 3D binary volume).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path may include, link or
 * call this file; only the tests, the package smoke check and the CPU
 * baseline of the benchmark use it.  It shares no code, header, table or
 * constant with the CUDA implementation.
 *
 * What it computes (the plain definition, not the paper's kernel steps):
 *   - A pixel P(x,y) has raster position x + y*W (Sec. 3, "Algorithm and
 *     implementation", first paragraph).  The row stride of the INPUT is
 *     `pitch` bytes; raster positions always use W.
 *   - I(x,y) = 1 is foreground, 0 background (same paragraph).  Any nonzero
 *     byte counts as foreground.
 *   - Adjacency: 4-connectivity (|dx|+|dy| == 1, the connectivity the paper
 *     evaluates, Sec. 4.3) or 8-connectivity (max(|dx|,|dy|) == 1).
 *   - The label of every pixel of a connected component C is
 *     1 + min over C of the raster position.  Background gets 0.  The paper's
 *     root is the element whose label equals its own address, and links
 *     always go from a larger to a smaller label (Sec. 3.1.1 and 3.1.3), so
 *     the root of a component is its smallest raster position; the +1 frees 0
 *     for the background.
 *
 * Two independent ways to reach that result are given:
 *   ccl_oracle_two_pass : classic raster two-pass union-find.
 *   ccl_oracle_bfs      : breadth-first flood fill started from each
 *                         unvisited foreground pixel in raster order (the
 *                         first pixel reached in raster order is the
 *                         component's minimum, so its index + 1 is the label).
 *
 * Both return 0 on success, 1 on invalid arguments, 2 when an allocation
 * fails.  H*W must stay below 2^31 - 1 so that 1 + index fits an int32.
 */
#include <stdint.h>
#include <stdlib.h>

static int args_ok(int64_t H, int64_t W, int64_t pitch, int conn)
{
    if (H < 0 || W < 0) return 0;
    if (H > 0 && W > 0 && pitch < W) return 0;
    if (conn != 4 && conn != 8) return 0;
    if (H * W > (int64_t)2147483646) return 0;
    return 1;
}

static int is_fg(const uint8_t *img, int64_t pitch, int64_t x, int64_t y)
{
    return img[y * pitch + x] != 0;
}

/* Root of x in the forest `parent`, halving the path on the way up. */
static int32_t uf_find(int32_t *parent, int32_t x)
{
    while (parent[x] != x) {
        parent[x] = parent[parent[x]];
        x = parent[x];
    }
    return x;
}

/* Join the trees of a and b; the larger root is hung under the smaller one,
 * so every root stays the smallest raster position of its tree. */
static void uf_union(int32_t *parent, int32_t a, int32_t b)
{
    int32_t ra = uf_find(parent, a);
    int32_t rb = uf_find(parent, b);
    if (ra == rb) return;
    if (ra < rb) parent[rb] = ra;
    else parent[ra] = rb;
}

int ccl_oracle_two_pass(const uint8_t *img, int64_t H, int64_t W, int64_t pitch,
                        int conn, int32_t *labels)
{
    if (!args_ok(H, W, pitch, conn)) return 1;
    int64_t N = H * W;
    if (N == 0) return 0;
    int32_t *parent = (int32_t *)malloc((size_t)N * sizeof(int32_t));
    if (!parent) return 2;

    /* Pass 1: every foreground pixel starts as its own tree (provisional
     * label = own position) and is joined with the foreground neighbours that
     * the raster scan has already visited: left and up for 4-connectivity,
     * plus up-left and up-right for 8-connectivity. */
    for (int64_t y = 0; y < H; ++y) {
        for (int64_t x = 0; x < W; ++x) {
            int32_t p = (int32_t)(y * W + x);
            if (!is_fg(img, pitch, x, y)) {
                parent[p] = -1;
                continue;
            }
            parent[p] = p;
            if (x > 0 && is_fg(img, pitch, x - 1, y))
                uf_union(parent, p, p - 1);
            if (y > 0 && is_fg(img, pitch, x, y - 1))
                uf_union(parent, p, (int32_t)(p - W));
            if (conn == 8 && y > 0) {
                if (x > 0 && is_fg(img, pitch, x - 1, y - 1))
                    uf_union(parent, p, (int32_t)(p - W - 1));
                if (x + 1 < W && is_fg(img, pitch, x + 1, y - 1))
                    uf_union(parent, p, (int32_t)(p - W + 1));
            }
        }
    }

    /* Pass 2: each foreground pixel takes 1 + its root. */
    for (int64_t p = 0; p < N; ++p)
        labels[p] = parent[p] < 0 ? 0 : uf_find(parent, (int32_t)p) + 1;

    free(parent);
    return 0;
}

int ccl_oracle_bfs(const uint8_t *img, int64_t H, int64_t W, int64_t pitch,
                   int conn, int32_t *labels)
{
    if (!args_ok(H, W, pitch, conn)) return 1;
    int64_t N = H * W;
    if (N == 0) return 0;
    int32_t *queue = (int32_t *)malloc((size_t)N * sizeof(int32_t));
    if (!queue) return 2;

    for (int64_t p = 0; p < N; ++p) labels[p] = 0;

    static const int dx8[8] = {-1, 1, 0, 0, -1, 1, -1, 1};
    static const int dy8[8] = {0, 0, -1, 1, -1, -1, 1, 1};
    int ndir = conn == 8 ? 8 : 4;

    for (int64_t y0 = 0; y0 < H; ++y0) {
        for (int64_t x0 = 0; x0 < W; ++x0) {
            int64_t seed = y0 * W + x0;
            if (!is_fg(img, pitch, x0, y0) || labels[seed] != 0) continue;
            /* seed is the first pixel of its component in raster order */
            int32_t lab = (int32_t)(seed + 1);
            int64_t head = 0, tail = 0;
            labels[seed] = lab;
            queue[tail++] = (int32_t)seed;
            while (head < tail) {
                int64_t q = queue[head++];
                int64_t qx = q % W, qy = q / W;
                for (int d = 0; d < ndir; ++d) {
                    int64_t nx = qx + dx8[d], ny = qy + dy8[d];
                    if (nx < 0 || ny < 0 || nx >= W || ny >= H) continue;
                    int64_t n = ny * W + nx;
                    if (!is_fg(img, pitch, nx, ny) || labels[n] != 0) continue;
                    labels[n] = lab;
                    queue[tail++] = (int32_t)n;
                }
            }
        }
    }
    free(queue);
    return 0;
}

/* ------------------------------------------------------------------------
 * 3D volumes.  The task the paper sets out (Sec. 1) is a unique ID per
 * connected region of a 2D or 3D image; its method is worked out in 2D.  The
 * volume extension reads the pixel model of Sec. 3 one dimension up:
 *   - voxel V(x,y,z) has raster position x + y*W + z*W*H; the INPUT has a
 *     row stride of `pitch` bytes and a slice stride of H*pitch bytes;
 *   - adjacency: 6-connectivity (|dx|+|dy|+|dz| == 1) or 26-connectivity
 *     (max(|dx|,|dy|,|dz|) == 1);
 *   - every voxel of a component C gets 1 + min over C of the raster
 *     position; background gets 0.
 * Same status codes as the 2D routines; D*H*W must stay below 2^31 - 1.
 */
static int args3_ok(int64_t D, int64_t H, int64_t W, int64_t pitch, int conn)
{
    if (D < 0 || H < 0 || W < 0) return 0;
    if (D > 0 && H > 0 && W > 0 && pitch < W) return 0;
    if (conn != 6 && conn != 26) return 0;
    if (D * H * W > (int64_t)2147483646) return 0;
    return 1;
}

static int is_fg3(const uint8_t *img, int64_t H, int64_t pitch, int64_t x, int64_t y, int64_t z)
{
    return img[(z * H + y) * pitch + x] != 0;
}

/* Is the offset (dx,dy,dz) a neighbour under `conn`? */
static int is_nbr3(int conn, int dx, int dy, int dz)
{
    int a = (dx < 0 ? -dx : dx) + (dy < 0 ? -dy : dy) + (dz < 0 ? -dz : dz);
    if (a == 0) return 0;
    return conn == 26 || a == 1;
}

int ccl_oracle3d_two_pass(const uint8_t *img, int64_t D, int64_t H, int64_t W, int64_t pitch,
                          int conn, int32_t *labels)
{
    if (!args3_ok(D, H, W, pitch, conn)) return 1;
    int64_t N = D * H * W;
    if (N == 0) return 0;
    int32_t *parent = (int32_t *)malloc((size_t)N * sizeof(int32_t));
    if (!parent) return 2;

    /* Pass 1 in raster order (x fastest, then y, then z): each foreground
     * voxel starts as its own tree and is joined with every foreground
     * neighbour that comes earlier in that order, i.e. the neighbours in the
     * previous slice, in the previous row of the same slice, and to the left. */
    for (int64_t z = 0; z < D; ++z) {
        for (int64_t y = 0; y < H; ++y) {
            for (int64_t x = 0; x < W; ++x) {
                int32_t p = (int32_t)((z * H + y) * W + x);
                if (!is_fg3(img, H, pitch, x, y, z)) {
                    parent[p] = -1;
                    continue;
                }
                parent[p] = p;
                for (int dz = -1; dz <= 0; ++dz) {
                    for (int dy = -1; dy <= 1; ++dy) {
                        for (int dx = -1; dx <= 1; ++dx) {
                            int earlier = dz < 0 || (dy < 0) || (dy == 0 && dx < 0);
                            if (!earlier || !is_nbr3(conn, dx, dy, dz)) continue;
                            int64_t nx = x + dx, ny = y + dy, nz = z + dz;
                            if (nx < 0 || ny < 0 || nz < 0 || nx >= W || ny >= H) continue;
                            if (!is_fg3(img, H, pitch, nx, ny, nz)) continue;
                            uf_union(parent, p, (int32_t)((nz * H + ny) * W + nx));
                        }
                    }
                }
            }
        }
    }

    /* Pass 2: each foreground voxel takes 1 + its root. */
    for (int64_t p = 0; p < N; ++p)
        labels[p] = parent[p] < 0 ? 0 : 1 + uf_find(parent, (int32_t)p);

    free(parent);
    return 0;
}

int ccl_oracle3d_bfs(const uint8_t *img, int64_t D, int64_t H, int64_t W, int64_t pitch,
                     int conn, int32_t *labels)
{
    if (!args3_ok(D, H, W, pitch, conn)) return 1;
    int64_t N = D * H * W;
    if (N == 0) return 0;
    int32_t *queue = (int32_t *)malloc((size_t)N * sizeof(int32_t));
    if (!queue) return 2;
    for (int64_t p = 0; p < N; ++p) labels[p] = 0;

    for (int64_t z0 = 0; z0 < D; ++z0) {
        for (int64_t y0 = 0; y0 < H; ++y0) {
            for (int64_t x0 = 0; x0 < W; ++x0) {
                int64_t seed = (z0 * H + y0) * W + x0;
                if (!is_fg3(img, H, pitch, x0, y0, z0) || labels[seed] != 0) continue;
                /* the first voxel of its component in raster order */
                int32_t lab = (int32_t)(seed + 1);
                int64_t head = 0, tail = 0;
                labels[seed] = lab;
                queue[tail++] = (int32_t)seed;
                while (head < tail) {
                    int64_t q = queue[head++];
                    int64_t qx = q % W, qy = (q / W) % H, qz = q / (W * H);
                    for (int dz = -1; dz <= 1; ++dz) {
                        for (int dy = -1; dy <= 1; ++dy) {
                            for (int dx = -1; dx <= 1; ++dx) {
                                if (!is_nbr3(conn, dx, dy, dz)) continue;
                                int64_t nx = qx + dx, ny = qy + dy, nz = qz + dz;
                                if (nx < 0 || ny < 0 || nz < 0 || nx >= W || ny >= H || nz >= D) continue;
                                int64_t n = (nz * H + ny) * W + nx;
                                if (!is_fg3(img, H, pitch, nx, ny, nz) || labels[n] != 0) continue;
                                labels[n] = lab;
                                queue[tail++] = (int32_t)n;
                            }
                        }
                    }
                }
            }
        }
    }
    free(queue);
    return 0;
}
