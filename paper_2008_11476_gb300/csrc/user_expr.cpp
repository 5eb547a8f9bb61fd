// User-defined point and local operators (Section 5.1: user kernels written
// against the framework's point / local abstractions are accelerated like the
// library's own nodes; here they become part of the kernel generated for
// their fused group).
//
// A user operator is an integer expression in a small C-like language:
//   expr    := or
//   or      := xor ('|' xor)*          xor := and ('^' and)*
//   and     := eq ('&' eq)*            eq  := rel (('==' | '!=') rel)*
//   rel     := shift (('<' | '>' | '<=' | '>=') shift)*
//   shift   := add (('<<' | '>>') add)*
//   add     := mul (('+' | '-') mul)*  mul := unary ('*' unary)*
//   unary   := ('-' | '+' | '~') unary | primary
//   primary := integer | a | b | c | in '(' int ',' int ')'
//            | (min | max) '(' expr ',' expr ')' | abs '(' expr ')' | '(' expr ')'
// with C precedence and 64-bit two's-complement arithmetic; comparisons give
// 0 or 1.  A point operator reads its inputs' values at the pixel as a, b, c;
// a local operator reads its input at literal offsets in(dx, dy) within its
// declared window, under its border mode.  The parser checks the grammar and
// the offsets and rewrites the expression into CUDA C++ (inputs become HVX_A,
// HVX_B, HVX_C and taps HVX_TAP(dx,dy), placeholders that the code generator
// replaces by its reads),
// so that nothing but these operations can reach the generated kernel.
#include <cctype>
#include <string>
#include <vector>

#include "hvx_internal.h"

namespace hvx {
namespace {

struct Parser {
    const std::string& s;
    size_t i = 0;
    bool local;
    int n_in, rx, ry;
    std::string out;
    std::string err;

    Parser(const std::string& src, bool loc, int n, int x, int y)
        : s(src), local(loc), n_in(n), rx(x), ry(y) {}

    void skip() {
        while (i < s.size() && std::isspace((unsigned char)s[i])) ++i;
    }
    bool peek(const char* t) {
        skip();
        return s.compare(i, std::char_traits<char>::length(t), t) == 0;
    }
    bool eat(const char* t) {
        if (!peek(t)) return false;
        i += std::char_traits<char>::length(t);
        return true;
    }
    bool fail(const std::string& m) {
        if (err.empty()) err = m + " at column " + std::to_string(i + 1);
        return false;
    }
    std::string ident() {
        skip();
        size_t j = i;
        while (j < s.size() && (std::isalnum((unsigned char)s[j]) || s[j] == '_')) ++j;
        if (j == i || std::isdigit((unsigned char)s[i])) return "";
        std::string id = s.substr(i, j - i);
        i = j;
        return id;
    }
    bool integer(long long* v) {
        skip();
        size_t j = i;
        while (j < s.size() && std::isdigit((unsigned char)s[j])) ++j;
        if (j == i || j - i > 18) return false;
        *v = std::stoll(s.substr(i, j - i));
        i = j;
        return true;
    }
    bool signed_int(int* v) {
        const bool neg = eat("-");
        long long x;
        if (!integer(&x) || x > 64) return false;
        *v = (int)(neg ? -x : x);
        return true;
    }

    // binary level with the given operators (longest first), then `next`
    template <class Next>
    bool level(const std::vector<const char*>& ops, Next next) {
        if (!next()) return false;
        for (;;) {
            const char* hit = nullptr;
            for (const char* op : ops)
                if (peek(op)) {
                    // '<' must not take '<<' / '<=', '&' not '&&', '|' not '||'
                    const size_t n = std::char_traits<char>::length(op);
                    const char after = i + n < s.size() ? s[i + n] : '\0';
                    if (n == 1 && (op[0] == '<' || op[0] == '>') && (after == op[0] || after == '='))
                        continue;
                    if (n == 1 && (op[0] == '&' || op[0] == '|') && after == op[0])
                        return fail("'&&' and '||' are not part of the language (use & and |)");
                    hit = op;
                    break;
                }
            if (!hit) return true;
            eat(hit);
            out += std::string(" ") + hit + " ";
            if (!next()) return false;
        }
    }

    bool expr() { return bor(); }
    bool bor() { return level({"|"}, [&] { return bxor(); }); }
    bool bxor() { return level({"^"}, [&] { return band(); }); }
    bool band() { return level({"&"}, [&] { return eq(); }); }
    bool eq() { return level({"==", "!="}, [&] { return rel(); }); }
    bool rel() { return level({"<=", ">=", "<", ">"}, [&] { return shift(); }); }
    bool shift() { return level({"<<", ">>"}, [&] { return add(); }); }
    bool add() { return level({"+", "-"}, [&] { return mul(); }); }
    bool mul() {
        if (peek("/") || peek("%")) return fail("division is not part of the language");
        return level({"*"}, [&] { return unary(); });
    }
    bool unary() {
        skip();
        if (peek("!") && !peek("!=")) return fail("'!' is not part of the language (use == 0)");
        if (eat("-")) {
            out += "(-";
            if (!unary()) return false;
            out += ")";
            return true;
        }
        if (eat("+")) return unary();
        if (eat("~")) {
            out += "(~";
            if (!unary()) return false;
            out += ")";
            return true;
        }
        return primary();
    }
    bool primary() {
        skip();
        if (i >= s.size()) return fail("expression ends early");
        if (eat("(")) {
            out += "(";
            if (!expr()) return false;
            if (!eat(")")) return fail("')' expected");
            out += ")";
            return true;
        }
        long long v;
        if (std::isdigit((unsigned char)s[i])) {
            if (!integer(&v)) return fail("integer literal too long");
            out += std::to_string(v) + "LL";
            return true;
        }
        const std::string id = ident();
        if (id.empty()) return fail("unexpected character");
        if (id == "a" || id == "b" || id == "c") {
            if (local) return fail("a local operator reads its input as in(dx, dy)");
            if (id[0] - 'a' >= n_in) return fail("'" + id + "' names no input");
            out += std::string("HVX_") + (char)std::toupper((unsigned char)id[0]);
            return true;
        }
        if (id == "in") {
            if (!local) return fail("in(dx, dy) is for local operators");
            int dx, dy;
            if (!eat("(") || !signed_int(&dx) || !eat(",") || !signed_int(&dy) || !eat(")"))
                return fail("in(dx, dy) takes two integer literals");
            if (dx < -rx || dx > rx || dy < -ry || dy > ry)
                return fail("offset outside the declared window");
            out += "HVX_TAP(" + std::to_string(dx) + "," + std::to_string(dy) + ")";
            return true;
        }
        if (id == "min" || id == "max") {
            out += "hvx_" + id + "(";
            if (!eat("(") || !expr() || !eat(",")) return fail(id + "(x, y) expected");
            out += ", ";
            if (!expr() || !eat(")")) return fail(id + "(x, y) expected");
            out += ")";
            return true;
        }
        if (id == "abs") {
            out += "hvx_abs(";
            if (!eat("(") || !expr() || !eat(")")) return fail("abs(x) expected");
            out += ")";
            return true;
        }
        return fail("unknown name '" + id + "'");
    }
};

}  // namespace

bool parse_user_expr(const std::string& src, bool local, int n_in, int rx, int ry,
                     std::string* code, std::string* why) {
    if (src.empty() || src.size() > 2048) {
        *why = "expression empty or longer than 2048 characters";
        return false;
    }
    Parser p(src, local, n_in, rx, ry);
    if (!p.expr()) {
        *why = p.err;
        return false;
    }
    p.skip();
    if (p.i != src.size()) {
        *why = "unexpected text at column " + std::to_string(p.i + 1);
        return false;
    }
    *code = p.out;
    return true;
}

}  // namespace hvx
