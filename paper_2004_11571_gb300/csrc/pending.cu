// Entry points whose implementations are not in this build yet.
#include "internal.h"

using namespace pe;

static pe_status not_built(const char *what)
{
    set_error("%s is not available in this build", what);
    return PE_ERR_ARG;
}

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
