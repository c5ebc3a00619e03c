/* The C ABI from plain C99 on a host-only context (no device touched): the
 * Section 2 vector-scaling example as chains of RW tasks over registered
 * buffers, submitted by pointer, plus the Section 3.2 error cases.  Exits 0
 * when the derived graph and the return codes are the expected ones. */
#include <errno.h>
#include <stdio.h>
#include <string.h>

#include "b3t.h"

#define CHECK(cond)                                                    \
    do {                                                               \
        if (!(cond)) {                                                 \
            fprintf(stderr, "failed: %s (line %d)\n", #cond, __LINE__); \
            return 1;                                                  \
        }                                                              \
    } while (0)

int main(void) {
    b3t_config cfg;
    memset(&cfg, 0, sizeof cfg);
    cfg.host_only = 1;
    b3t_ctx *ctx = NULL;
    CHECK(b3t_init(&ctx, &cfg, NULL) == 0);

    /* four 16-byte aligned stand-in buffers, never dereferenced */
    void *blk[4];
    b3t_handle h[4];
    for (int i = 0; i < 4; ++i) {
        blk[i] = (void *)(uintptr_t)(0x10000000u + ((uintptr_t)i << 20));
        CHECK(b3t_data_register(ctx, blk[i], 1024, 4, 0, &h[i]) == 0);
    }
    const uint8_t rw[1] = {B3T_RW};
    b3t_codelet scal;
    CHECK(b3t_task_decl(ctx, "scale_vector", B3T_SCAL_F32, 1, rw, sizeof(float), &scal) == 0);

    /* three factors per block, level by level: 12 tasks, one chain per block */
    const float f[3] = {2.0f, 0.5f, 3.0f};
    for (int k = 0; k < 3; ++k)
        for (int i = 0; i < 4; ++i) CHECK(b3t_task_submit_ptrs(ctx, scal, &blk[i], 1, &f[k], sizeof f[k]) == 0);
    int64_t nt = 0, ne = 0;
    CHECK(b3t_dag_stats(ctx, &nt, &ne) == 0);
    CHECK(nt == 12 && ne == 8);
    int32_t pred[8], succ[8];
    int64_t count = 0;
    CHECK(b3t_dag_edges(ctx, pred, succ, 8, &count) == 0 && count == 8);
    for (int e = 0; e < 8; ++e) CHECK(succ[e] == pred[e] + 4);   /* task (k, i) -> (k + 1, i) */

    /* Section 3.2 diagnostics as return codes */
    void *unregistered = (void *)(uintptr_t)0x7f000000u;
    CHECK(b3t_task_submit_ptrs(ctx, scal, &unregistered, 1, &f[0], sizeof f[0]) == -ENOENT);
    CHECK(b3t_task_submit_ptrs(ctx, scal, &blk[0], 1, &f[0], 2) == -EINVAL);     /* wrong scalar size */
    const uint8_t r[1] = {B3T_R};
    CHECK(b3t_task_submit(ctx, scal, &h[0], r, 1, &f[0], sizeof f[0]) == -EINVAL);  /* mode mismatch */
    CHECK(b3t_data_register(ctx, blk[0], 1024, 4, 0, &h[0]) == -EEXIST);
    CHECK(b3t_strerror(-ENOENT) != NULL && strlen(b3t_strerror(-ENOENT)) > 0);
    CHECK(b3t_task_wait(ctx, 0) == -ENODEV);                      /* host-only: nothing runs */

    CHECK(b3t_shutdown(ctx) == 0);
    printf("c abi ok\n");
    return 0;
}
