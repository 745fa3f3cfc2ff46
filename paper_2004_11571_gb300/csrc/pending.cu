// Entry points whose implementations are not in this build yet.
#include "internal.h"

using namespace pe;

static pe_status not_built(const char *what)
{
    set_error("%s is not available in this build", what);
    return PE_ERR_ARG;
}

extern "C" pe_status poly_eval_batch_plan(const pe_job *, size_t, pe_batch **out)
{
    if (out) *out = nullptr;
    return not_built("poly_eval_batch_plan");
}
extern "C" pe_status poly_eval_batch_launch(pe_batch *, void *) { return not_built("poly_eval_batch_launch"); }
extern "C" pe_status poly_eval_batch_set_beta(pe_batch *, size_t, const uint64_t *) { return not_built("poly_eval_batch_set_beta"); }
extern "C" void poly_eval_batch_destroy(pe_batch *) {}
extern "C" pe_status poly_eval_batch(const pe_job *, size_t, void *) { return not_built("poly_eval_batch"); }
extern "C" pe_status poly_eval_tune(pe_poly *, uint64_t, pe_tiles *, double *) { return not_built("poly_eval_tune"); }
extern "C" pe_status poly_eval_tune_save(const char *) { return not_built("poly_eval_tune_save"); }
extern "C" pe_status poly_eval_tune_load(const char *) { return not_built("poly_eval_tune_load"); }
extern "C" pe_status poly_eval_server_create(const pe_server_cfg *, pe_server **out)
{
    if (out) *out = nullptr;
    return not_built("poly_eval_server_create");
}
extern "C" pe_status poly_eval_server_register(pe_server *, const pe_poly_desc *, uint64_t *) { return not_built("server"); }
extern "C" pe_status poly_eval_server_submit(pe_server *, const pe_request *, uint64_t *) { return not_built("server"); }
extern "C" pe_status poly_eval_server_poll(pe_server *, uint64_t, int64_t) { return not_built("server"); }
extern "C" pe_status poly_eval_server_stats(pe_server *, pe_server_stats *) { return not_built("server"); }
extern "C" void poly_eval_server_destroy(pe_server *) {}
