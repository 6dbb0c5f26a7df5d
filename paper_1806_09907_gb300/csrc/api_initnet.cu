// C ABI of the learned initialisation: convolution layers, the network's
// glue kernels, the field loss, flat Adam and the training-volume renderer.
// Declarations and contracts: include/airgb.h.
#include "airgb.h"
#include "checks.h"
#include "launch.h"

using namespace airgb;

namespace {

cudaStream_t St(al_stream s) { return (cudaStream_t)s; }

constexpr int64_t kMaxRows = ((int64_t)1 << 31) - 1;

al_status check_conv(const al_conv3d *cv, ConvLayer *l)
{
    if (!cv)
        return AL_ERR_INVALID_ARG;
    if (cv->batch < 1 || (cv->stride != 1 && cv->stride != 2))
        return AL_ERR_INVALID_ARG;
    if (!(cv->cin == 2 || (cv->cin % 8 == 0 && cv->cin >= 8 && cv->cin <= 256)))
        return AL_ERR_SHAPE;
    if (cv->cout % 16 != 0 || cv->cout < 16 || cv->cout > 128)
        return AL_ERR_SHAPE;
    for (int k = 0; k < 3; ++k)
        if (cv->size[k] < 1 || cv->size[k] > (1 << 20))
            return AL_ERR_SHAPE;
    const int64_t vin = (int64_t)cv->batch * cv->size[0] * cv->size[1] * cv->size[2];
    if (vin > kMaxRows)
        return AL_ERR_SHAPE;
    // the kernels keep tap offsets (up to 3 planes of a volume's channels) in
    // 32-bit integers
    const int64_t plane_in = cv->size[1] * cv->size[2] * (int64_t)cv->cin;
    const int64_t ho = (cv->size[1] - 1) / cv->stride + 1, wo = (cv->size[2] - 1) / cv->stride + 1;
    if (3 * plane_in >= kMaxRows || 3 * ho * wo * (int64_t)cv->cout >= kMaxRows)
        return AL_ERR_SHAPE;
    l->nb = cv->batch;
    l->D = (int)cv->size[0];
    l->H = (int)cv->size[1];
    l->W = (int)cv->size[2];
    l->cin = cv->cin;
    l->cout = cv->cout;
    l->stride = cv->stride;
    return AL_OK;
}

al_status ok_launch(cudaError_t e) { return e == cudaSuccess ? AL_OK : AL_ERR_CUDA; }

al_status check_net(int32_t batch, const int64_t *n3, NetGrid *g)
{
    if (batch < 1 || !n3)
        return AL_ERR_INVALID_ARG;
    int64_t v = batch;
    for (int k = 0; k < 3; ++k) {
        if (n3[k] < 1 || n3[k] > (1 << 16))
            return AL_ERR_SHAPE;
        v *= n3[k];
    }
    if (v * 256 > kMaxRows * 64)
        return AL_ERR_SHAPE;
    g->nb = batch;
    for (int k = 0; k < 3; ++k) {
        g->n3[k] = (int)n3[k];
        g->n4[k] = (int)((n3[k] - 1) / 2 + 1);
    }
    return AL_OK;
}

}  // namespace

extern "C" {

al_status al_conv3d_output_size(const al_conv3d *cv, int64_t *out)
{
    ConvLayer l;
    const al_status st = check_conv(cv, &l);
    if (st != AL_OK)
        return st;
    if (!out)
        return AL_ERR_INVALID_ARG;
    for (int k = 0; k < 3; ++k)
        out[k] = (cv->size[k] - 1) / cv->stride + 1;
    return AL_OK;
}

size_t al_conv3d_packed_bytes(const al_conv3d *cv, int32_t dgrad)
{
    ConvLayer l;
    if (check_conv(cv, &l) != AL_OK)
        return 0;
    if (dgrad && l.cin % 16 != 0)
        return 0;
    return conv_packed_elems(l, dgrad ? 1 : 0) * 2;
}

al_status al_conv3d_pack(const al_conv3d *cv, const float *weight, void *packed_fwd,
                         void *packed_dgrad, al_stream stream)
{
    ConvLayer l;
    al_status st = check_conv(cv, &l);
    if (st != AL_OK)
        return st;
    if (!weight || (!packed_fwd && !packed_dgrad))
        return AL_ERR_INVALID_ARG;
    if (packed_dgrad && (l.cin % 16 != 0 || l.cin > 128))
        return AL_ERR_UNSUPPORTED;
    if (!aligned16(weight) || !aligned16(packed_fwd) || !aligned16(packed_dgrad))
        return AL_ERR_ALIGN;
    return ok_launch(launch_conv_pack(l, weight, packed_fwd, packed_dgrad, St(stream)));
}

size_t al_conv3d_forward_workspace_bytes(const al_conv3d *cv)
{
    ConvLayer l;
    if (check_conv(cv, &l) != AL_OK)
        return 0;
    return conv_fwd_ws_bytes(l);
}

al_status al_conv3d_forward(const al_conv3d *cv, const void *input, const void *packed_fwd,
                            const float *bias, int32_t relu, int32_t out_f32, void *output,
                            void *workspace, size_t workspace_bytes, al_stream stream)
{
    ConvLayer l;
    al_status st = check_conv(cv, &l);
    if (st != AL_OK)
        return st;
    if (!input || !packed_fwd || !output)
        return AL_ERR_INVALID_ARG;
    const int64_t vout = (int64_t)l.nb * conv_out_size(l.D, l.stride) *
                         conv_out_size(l.H, l.stride) * conv_out_size(l.W, l.stride);
    if (vout > kMaxRows)
        return AL_ERR_SHAPE;
    if (!aligned16(input) || !aligned16(packed_fwd) || !aligned16(output) || !aligned16(bias) ||
        !aligned16(workspace))
        return AL_ERR_ALIGN;
    // a workspace too small for the split-K partials runs the layer unsplit
    void *ws = workspace && workspace_bytes >= conv_fwd_ws_bytes(l) && conv_fwd_ws_bytes(l) > 0
                   ? workspace
                   : nullptr;
    return ok_launch(launch_conv_forward(l, input, packed_fwd, bias, relu ? 1 : 0,
                                         out_f32 ? 1 : 0, output, ws, St(stream)));
}

al_status al_conv3d_backward_data(const al_conv3d *cv, const void *grad_output,
                                  const void *packed_dgrad, const void *relu_input,
                                  const void *addend, int32_t addend_stride,
                                  int32_t addend_offset, void *grad_input, al_stream stream)
{
    ConvLayer l;
    al_status st = check_conv(cv, &l);
    if (st != AL_OK)
        return st;
    if (!grad_output || !packed_dgrad || !grad_input)
        return AL_ERR_INVALID_ARG;
    if (l.cin % 16 != 0 || l.cin > 128)
        return AL_ERR_UNSUPPORTED;
    if (addend && (addend_stride < l.cin || addend_offset < 0 ||
                   addend_offset + l.cin > addend_stride || addend_stride % 8 != 0 ||
                   addend_offset % 8 != 0))
        return AL_ERR_INVALID_ARG;
    if (!aligned16(grad_output) || !aligned16(packed_dgrad) || !aligned16(grad_input) ||
        !aligned16(relu_input) || !aligned16(addend))
        return AL_ERR_ALIGN;
    return ok_launch(launch_conv_dgrad(l, grad_output, packed_dgrad, relu_input, addend,
                                       addend_stride, addend_offset, grad_input, St(stream)));
}

size_t al_conv3d_backward_weight_workspace_bytes(const al_conv3d *cv)
{
    ConvLayer l;
    if (check_conv(cv, &l) != AL_OK)
        return 0;
    return conv_wgrad_ws_bytes(l);
}

al_status al_conv3d_backward_weight(const al_conv3d *cv, const void *input,
                                    const void *grad_output, float *grad_weight, float *grad_bias,
                                    void *workspace, size_t workspace_bytes, al_stream stream)
{
    ConvLayer l;
    al_status st = check_conv(cv, &l);
    if (st != AL_OK)
        return st;
    if (!input || !grad_output || !grad_weight)
        return AL_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < conv_wgrad_ws_bytes(l))
        return AL_ERR_WORKSPACE;
    if (!aligned16(input) || !aligned16(grad_output) || !aligned16(workspace))
        return AL_ERR_ALIGN;
    return ok_launch(
        launch_conv_wgrad(l, input, grad_output, grad_weight, grad_bias, workspace, St(stream)));
}

al_status al_initnet_input(int32_t batch, const int64_t *size, const float *fixed,
                           const float *moving, void *x, al_stream stream)
{
    if (batch < 1 || !size || !fixed || !moving || !x)
        return AL_ERR_INVALID_ARG;
    int64_t n = batch;
    for (int k = 0; k < 3; ++k) {
        if (size[k] < 1)
            return AL_ERR_SHAPE;
        n *= size[k];
    }
    if (n > kMaxRows)
        return AL_ERR_SHAPE;
    if (!aligned16(fixed) || !aligned16(moving) || !aligned16(x))
        return AL_ERR_ALIGN;
    return ok_launch(launch_net_input(n, fixed, moving, x, St(stream)));
}

al_status al_initnet_upcat(int32_t batch, const int64_t *n3, int32_t c4, int32_t c3,
                           const void *e4, const void *e3, void *cat, al_stream stream)
{
    NetGrid g;
    al_status st = check_net(batch, n3, &g);
    if (st != AL_OK)
        return st;
    if (!e4 || !e3 || !cat || c4 < 8 || c3 < 8 || c4 % 8 || c3 % 8)
        return AL_ERR_INVALID_ARG;
    if (!aligned16(e4) || !aligned16(e3) || !aligned16(cat))
        return AL_ERR_ALIGN;
    return ok_launch(launch_upcat(g, c4, c3, e4, e3, cat, St(stream)));
}

al_status al_initnet_upcat_adjoint(int32_t batch, const int64_t *n3, int32_t c4, int32_t c3,
                                   const void *grad_cat, const void *e4, void *grad_e4,
                                   al_stream stream)
{
    NetGrid g;
    al_status st = check_net(batch, n3, &g);
    if (st != AL_OK)
        return st;
    if (!grad_cat || !e4 || !grad_e4 || c4 < 8 || c3 < 8 || c4 % 8 || c3 % 8)
        return AL_ERR_INVALID_ARG;
    if (!aligned16(grad_cat) || !aligned16(e4) || !aligned16(grad_e4))
        return AL_ERR_ALIGN;
    return ok_launch(launch_upcat_adjoint(g, c4, c3, grad_cat, e4, grad_e4, St(stream)));
}

static al_status net_lattice(const al_bspline *bs, int32_t batch, const int64_t *n3,
                             int32_t channels, NetGrid *g)
{
    al_status st = check_net(batch, n3, g);
    if (st != AL_OK)
        return st;
    Grid gr;
    Lattice L;
    st = check_bspline(bs, &gr, &L);
    if (st != AL_OK)
        return st;
    if (bs->grid.ndim != 3 || channels < 3 || channels % 4 != 0)
        return AL_ERR_SHAPE;
    // the head sits at every 8th voxel: n3 = (N - 1)/8 + 1 per axis
    if (bs->spacing != 8)
        return AL_ERR_UNSUPPORTED;
    for (int k = 0; k < 3; ++k)
        if (n3[2 - k] != (bs->grid.size[k] - 1) / 8 + 1)
            return AL_ERR_SHAPE;
    g->lat[0] = L.nx;
    g->lat[1] = L.ny;
    g->lat[2] = L.nz;
    return AL_OK;
}

al_status al_initnet_head_to_ctrl(const al_bspline *bs, int32_t batch, const int64_t *n3,
                                  int32_t channels, const float *head, float *ctrl,
                                  al_stream stream)
{
    NetGrid g;
    al_status st = net_lattice(bs, batch, n3, channels, &g);
    if (st != AL_OK)
        return st;
    if (!head || !ctrl)
        return AL_ERR_INVALID_ARG;
    if (!aligned16(head) || !aligned16(ctrl))
        return AL_ERR_ALIGN;
    return ok_launch(launch_head_to_ctrl(g, channels, head, ctrl, St(stream)));
}

al_status al_initnet_head_adjoint(const al_bspline *bs, int32_t batch, const int64_t *n3,
                                  int32_t channels, const float *grad_ctrl, void *grad_head,
                                  al_stream stream)
{
    NetGrid g;
    al_status st = net_lattice(bs, batch, n3, channels, &g);
    if (st != AL_OK)
        return st;
    if (!grad_ctrl || !grad_head)
        return AL_ERR_INVALID_ARG;
    if (!aligned16(grad_ctrl) || !aligned16(grad_head))
        return AL_ERR_ALIGN;
    return ok_launch(launch_head_adjoint(g, channels, grad_ctrl, grad_head, St(stream)));
}

size_t al_field_loss_workspace_bytes(int32_t batch)
{
    return batch < 1 ? 0 : (size_t)batch * 3 * sizeof(double);
}

al_status al_field_loss(const al_bspline *bs, int32_t batch, const float *ctrl,
                        const float *ctrl_true, double *loss_dev, float *grad_ctrl,
                        void *workspace, size_t workspace_bytes, al_stream stream)
{
    Grid g;
    Lattice L;
    al_status st = check_bspline(bs, &g, &L);
    if (st != AL_OK)
        return st;
    if (bs->grid.ndim != 3)
        return AL_ERR_SHAPE;
    if (batch < 1 || !ctrl || !ctrl_true || !loss_dev || !grad_ctrl)
        return AL_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < al_field_loss_workspace_bytes(batch))
        return AL_ERR_WORKSPACE;
    if (!aligned16(ctrl) || !aligned16(ctrl_true) || !aligned16(grad_ctrl) ||
        !aligned16(workspace))
        return AL_ERR_ALIGN;
    FieldLossArgs a;
    a.n[0] = L.nx;
    a.n[1] = L.ny;
    a.n[2] = L.nz;
    a.N[0] = g.X;
    a.N[1] = g.Y;
    a.N[2] = g.Z;
    a.delta = L.delta;
    const double nv = (double)g.nv;
    a.gscale = 2.0 / (3.0 * nv * batch);
    a.lscale = 1.0 / (3.0 * nv * batch);
    if (field_loss_smem(a) > 200 * 1024)
        return AL_ERR_UNSUPPORTED;
    return ok_launch(launch_field_loss(a, batch, ctrl, ctrl_true, grad_ctrl,
                                       static_cast<double *>(workspace), loss_dev, St(stream)));
}

al_status al_adam_flat(const al_adam_params *p, int64_t n, int64_t *step, float *param,
                       const float *grad, float *m, float *v, al_stream stream)
{
    if (!p || n < 1 || !step || !param || !grad || !m || !v)
        return AL_ERR_INVALID_ARG;
    if (!(p->lr > 0) || !(p->beta1 >= 0 && p->beta1 < 1) || !(p->beta2 >= 0 && p->beta2 < 1) ||
        !(p->eps >= 0))
        return AL_ERR_INVALID_ARG;
    if (!aligned16(param) || !aligned16(grad) || !aligned16(m) || !aligned16(v))
        return AL_ERR_ALIGN;
    AdamFlatArgs a;
    a.beta1 = p->beta1;
    a.beta2 = p->beta2;
    a.lr = (float)p->lr;
    a.eps = (float)p->eps;
    a.n = n;
    return ok_launch(launch_adam_flat(a, step, param, grad, m, v, St(stream)));
}

al_status al_adam_flat_pack(const al_adam_params *p, int64_t n, int64_t *step, float *param,
                            const float *grad, float *m, float *v, int32_t n_layers,
                            const al_conv3d *layers, const int64_t *weight_offset,
                            void *const *packed_fwd, void *const *packed_dgrad, al_stream stream)
{
    if (!p || n < 1 || !step || !param || !grad || !m || !v)
        return AL_ERR_INVALID_ARG;
    if (!(p->lr > 0) || !(p->beta1 >= 0 && p->beta1 < 1) || !(p->beta2 >= 0 && p->beta2 < 1) ||
        !(p->eps >= 0))
        return AL_ERR_INVALID_ARG;
    if (n_layers < 1 || n_layers > kMaxPackLayers || !layers || !weight_offset || !packed_fwd ||
        !packed_dgrad)
        return AL_ERR_INVALID_ARG;
    if (!aligned16(param) || !aligned16(grad) || !aligned16(m) || !aligned16(v))
        return AL_ERR_ALIGN;
    AdamPackArgs a = {};
    a.adam.beta1 = p->beta1;
    a.adam.beta2 = p->beta2;
    a.adam.lr = (float)p->lr;
    a.adam.eps = (float)p->eps;
    a.adam.n = n;
    a.nl = n_layers;
    int64_t lo[kMaxPackLayers], hi[kMaxPackLayers];
    for (int j = 0; j < n_layers; ++j) {
        ConvLayer l;
        const al_status st = check_conv(&layers[j], &l);
        if (st != AL_OK)
            return st;
        void *pf = packed_fwd[j], *pd = packed_dgrad[j];
        if (!pf && !pd)
            return AL_ERR_INVALID_ARG;
        if (pd && (l.cin % 16 != 0 || l.cin > 128))
            return AL_ERR_UNSUPPORTED;
        if (!aligned16(pf) || !aligned16(pd))
            return AL_ERR_ALIGN;
        lo[j] = weight_offset[j];
        hi[j] = lo[j] + (int64_t)l.cout * 27 * l.cin;
        if (lo[j] < 0 || hi[j] > n)
            return AL_ERR_INVALID_ARG;
        for (int i = 0; i < j; ++i)
            if (lo[j] < hi[i] && lo[i] < hi[j])
                return AL_ERR_INVALID_ARG;  // weight ranges overlap
        adam_pack_layer(l, lo[j], pf, pd, &a.L[j]);
    }
    return ok_launch(launch_adam_pack(a, step, param, grad, m, v, St(stream)));
}

al_status al_render_blobs(const int64_t *size, int32_t count, int32_t n_blobs, const float *table,
                          float *out, al_stream stream)
{
    if (!size || count < 1 || count > 65535 || n_blobs < 1 || n_blobs > 1024 || !table || !out)
        return AL_ERR_INVALID_ARG;
    int64_t nv = 1;
    for (int k = 0; k < 3; ++k) {
        if (size[k] < 1 || size[k] > (1 << 16))
            return AL_ERR_SHAPE;
        nv *= size[k];
    }
    if (nv * count > ((int64_t)1 << 40))
        return AL_ERR_SHAPE;
    if (!aligned16(table) || !aligned16(out))
        return AL_ERR_ALIGN;
    return ok_launch(launch_render_blobs((int)size[0], (int)size[1], (int)size[2], count, n_blobs,
                                         table, out, St(stream)));
}

}  // extern "C"
